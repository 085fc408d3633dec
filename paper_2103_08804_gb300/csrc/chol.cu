// Direct shifted solve (S + lambda I) x = F of the natural-gradient update
// (Sec. III) for large P: blocked right-looking Cholesky S = L L^dag on many
// CTAs, then iterative refinement in float64.
//
// S (float64, full Hermitian, shift on its diagonal) stays untouched; its
// lower triangle is copied into the factor buffer L in the factor precision
// (float64 for float64 contexts, float32 otherwise) and factored in place in
// 64 x 64 blocks.  Per block column J:
//   potrf_kernel   L_JJ = chol(A_JJ)                   (one CTA, in shared memory)
//   trsm_kernel    L_IJ = A_IJ L_JJ^{-dag}, I > J      (one warp per row)
//   syrk_kernel    A_IK -= L_IJ L_KJ^dag, J < K <= I   (one CTA per 64 x 64 block)
// The solve with a float32 factor (and float32 arithmetic in the triangular
// solves) is accurate to about kappa * 2^-24, so it is refined in float64
// (Wilkinson's iterative refinement; the residual is formed in float64):
//   x = 0, r = F;  repeat { d = L^{-dag} L^{-1} r;  x += d;  r = F - S x }
// until |r| <= REFINE_TOL |F|, the residual stops shrinking (by 2x), or
// REFINE_MAXIT steps.  A float64 factor needs one step.  The triangular
// solves run one 64-row block column per launch; every later launch of a
// refinement step returns at once when the done flag is set, so the launch
// sequence is fixed (graph-capturable).
#include "common.cuh"

namespace {

constexpr int NB = 64;
constexpr int NTRI = NB * (NB + 1) / 2;
constexpr int REFINE_MAXIT = 10;
constexpr double REFINE_TOL = 1e-12;
constexpr int RES_GRID = 304;  // CTAs of the residual kernel (fixed: deterministic sums)

CR_HD int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <typename R> CR_D cpx<R> shfl(cpx<R> v, int src) {
    return {__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src)};
}

// L <- S in the factor precision (whole matrix; only the lower triangle is used).
template <typename R>
__global__ void chol_copy_kernel(const double* __restrict__ S_, int P, cpx<R>* __restrict__ L) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (size_t)P * P) L[idx] = ccast<R>(((const cpx<double>*)S_)[idx]);
}

// Factor the diagonal block J in shared memory (packed lower triangle, in
// the factor precision: float64 is a narrow pipe on this GPU and the
// float64 refinement corrects the float32 factor anyway); zero its strict
// upper part.  A non-positive pivot sets CR_ESINGULAR and is replaced by 1
// so the factorisation runs to the end.
template <typename R>
__global__ void __launch_bounds__(256) potrf_kernel(cpx<R>* __restrict__ L, int P, int J,
                                                    int* __restrict__ status) {
    __shared__ cpx<R> a[NTRI];
    __shared__ R piv;
    __shared__ int bad;
    const int base = J * NB, n = min(NB, P - base), t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (j <= i) a[tri(i, j)] = L[(size_t)(base + i) * P + base + j];
    }
    for (int j = 0; j < n; ++j) {
        __syncthreads();
        if (t == 0) {
            R d = a[tri(j, j)].x;
            if (!(d > R(0))) {
                bad = 1;
                d = R(1);
            }
            piv = m_sqrt(d);
            a[tri(j, j)] = {piv, R(0)};
        }
        __syncthreads();
        const R ip = R(1) / piv;
        for (int i = j + 1 + t; i < n; i += blockDim.x) a[tri(i, j)] = ip * a[tri(i, j)];
        __syncthreads();
        const int m = n - j - 1;
        for (int e = t; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e / m, l = j + 1 + e % m;
            if (l <= i) a[tri(i, l)] = a[tri(i, l)] - a[tri(i, j)] * conj(a[tri(l, j)]);
        }
    }
    __syncthreads();
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        L[(size_t)(base + i) * P + base + j] = j <= i ? a[tri(i, j)] : cpx<R>{R(0), R(0)};
    }
    if (t == 0 && bad) set_status(status, CR_ESINGULAR);
}

// Rows below block J (block J is full here: it is not the last block):
// x L_JJ^dag = a solved column by column, lanes holding columns lane and
// lane + 32 of one row.
template <typename R>
__global__ void __launch_bounds__(256) trsm_kernel(cpx<R>* __restrict__ L, int P, int J) {
    __shared__ cpx<R> d[NTRI];
    const int base = J * NB, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int e = t; e < NB * NB; e += blockDim.x) {
        const int i = e / NB, j = e % NB;
        if (j <= i) d[tri(i, j)] = L[(size_t)(base + i) * P + base + j];
    }
    __syncthreads();
    for (int row = base + NB + blockIdx.x * 8 + warp; row < P; row += gridDim.x * 8) {
        cpx<R>* Lr = L + (size_t)row * P + base;
        cpx<R> v0 = Lr[lane], v1 = Lr[lane + 32];
        for (int c = 0; c < NB; ++c) {
            cpx<R> xc = shfl(c < 32 ? v0 : v1, c & 31);
            xc = (R(1) / d[tri(c, c)].x) * xc;
            if (lane == (c & 31)) {
                if (c < 32) v0 = xc;
                else v1 = xc;
            }
            if (lane > c) v0 = v0 - xc * conj(d[tri(lane, c)]);
            if (lane + 32 > c) v1 = v1 - xc * conj(d[tri(lane + 32, c)]);
        }
        Lr[lane] = v0;
        Lr[lane + 32] = v1;
    }
}

// Trailing update of the lower block pairs (I, K), J < K <= I, one CTA per
// pair (linear index -> row a = I - J - 1, column b = K - J - 1 with b <= a);
// 16 x 16 threads, 4 x 4 outputs each (rows ty + 16 q, columns tx + 16 q).
template <typename R>
__global__ void __launch_bounds__(256) syrk_kernel(cpx<R>* __restrict__ L, int P, int J) {
    constexpr int KC = 16;
    __shared__ cpx<R> As[KC][NB + 1], Bs[KC][NB + 1];
    const long long idx = blockIdx.x;
    int a = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
    while ((long long)a * (a + 1) / 2 > idx) --a;
    while ((long long)(a + 1) * (a + 2) / 2 <= idx) ++a;
    const int b = (int)(idx - (long long)a * (a + 1) / 2);
    const int i0 = (J + 1 + a) * NB, k0 = (J + 1 + b) * NB, c0 = J * NB;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    cpx<R> acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) acc[q][q2] = {R(0), R(0)};
    for (int cc = 0; cc < NB; cc += KC) {
        for (int e = threadIdx.x; e < NB * KC; e += blockDim.x) {
            const int r = e / KC, c = e % KC, gi = i0 + r, gk = k0 + r;
            As[c][r] = gi < P ? L[(size_t)gi * P + c0 + cc + c] : cpx<R>{R(0), R(0)};
            Bs[c][r] = gk < P ? L[(size_t)gk * P + c0 + cc + c] : cpx<R>{R(0), R(0)};
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            cpx<R> av[4], bv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                av[q] = As[c][ty + 16 * q];
                bv[q] = conj(Bs[c][tx + 16 * q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int q2 = 0; q2 < 4; ++q2) acc[q][q2] = acc[q][q2] + av[q] * bv[q2];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int q2 = 0; q2 < 4; ++q2) {
            const int i = i0 + ty + 16 * q, k = k0 + tx + 16 * q2;
            if (i < P && k < P) {
                cpx<R>* p = L + (size_t)i * P + k;
                *p = *p - acc[q][q2];
            }
        }
}

// Block column J of L y = r: every CTA stages L_JJ in shared memory and
// solves y_J = L_JJ^{-1} r_J (warp 0), CTA 0 stores it; rows below get
// r_i -= L_iJ y_J (one warp per row).  r is scratch (overwritten below
// block J), y the result.
template <typename R>
__global__ void __launch_bounds__(256) trsv_fwd_kernel(const cpx<R>* __restrict__ L, int P, int J,
                                                       double* __restrict__ r_,
                                                       double* __restrict__ y_,
                                                       const double* __restrict__ skip) {
    if (*skip != 0.0) return;
    __shared__ cpx<R> d[NTRI];
    __shared__ cpx<R> ys[NB];
    cpx<double>* r = (cpx<double>*)r_;
    cpx<double>* y = (cpx<double>*)y_;
    const int base = J * NB, n = min(NB, P - base), t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (j <= i) d[tri(i, j)] = L[(size_t)(base + i) * P + base + j];
    }
    __syncthreads();
    if (warp == 0) {
        const cpx<R> z = {R(0), R(0)};
        cpx<R> v0 = lane < n ? ccast<R>(r[base + lane]) : z;
        cpx<R> v1 = lane + 32 < n ? ccast<R>(r[base + lane + 32]) : z;
        for (int c = 0; c < n; ++c) {
            cpx<R> yc = shfl(c < 32 ? v0 : v1, c & 31);
            yc = (R(1) / d[tri(c, c)].x) * yc;
            if (lane == (c & 31)) {
                if (c < 32) v0 = yc;
                else v1 = yc;
            }
            if (lane > c && lane < n) v0 = v0 - d[tri(lane, c)] * yc;
            if (lane + 32 > c && lane + 32 < n) v1 = v1 - d[tri(lane + 32, c)] * yc;
        }
        if (lane < n) ys[lane] = v0;
        if (lane + 32 < n) ys[lane + 32] = v1;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int e = t; e < n; e += blockDim.x) y[base + e] = ccast<double>(ys[e]);
    for (int row = base + n + blockIdx.x * 8 + warp; row < P; row += gridDim.x * 8) {
        const cpx<R>* Lr = L + (size_t)row * P + base;
        cpx<R> s = Lr[lane] * ys[lane];
        s = s + Lr[lane + 32] * ys[lane + 32];
        s = warp_sum(s);
        if (lane == 0) r[row] = r[row] - ccast<double>(s);
    }
}

// Block column J of L^dag x = y (J descending): every CTA stages L_JJ in
// shared memory and solves x_J = L_JJ^{-dag} y_J (warp 0), CTA 0 stores it;
// the 32 rows i above the block that a CTA owns get
// y_i -= sum_c conj(L_{base + c, i}) x_c (lanes along i, warps along c).
template <typename R>
__global__ void __launch_bounds__(256) trsv_bwd_kernel(const cpx<R>* __restrict__ L, int P, int J,
                                                       double* __restrict__ y_,
                                                       double* __restrict__ x_,
                                                       const double* __restrict__ skip) {
    if (*skip != 0.0) return;
    __shared__ cpx<R> d[NTRI];
    __shared__ cpx<R> xs[NB];
    cpx<double>* y = (cpx<double>*)y_;
    cpx<double>* x = (cpx<double>*)x_;
    const int base = J * NB, n = min(NB, P - base), t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int e = t; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        if (j <= i) d[tri(i, j)] = L[(size_t)(base + i) * P + base + j];
    }
    __syncthreads();
    if (warp == 0) {
        const cpx<R> z = {R(0), R(0)};
        cpx<R> v0 = lane < n ? ccast<R>(y[base + lane]) : z;
        cpx<R> v1 = lane + 32 < n ? ccast<R>(y[base + lane + 32]) : z;
        for (int c = n - 1; c >= 0; --c) {
            cpx<R> xc = shfl(c < 32 ? v0 : v1, c & 31);
            xc = (R(1) / d[tri(c, c)].x) * xc;
            if (lane == (c & 31)) {
                if (c < 32) v0 = xc;
                else v1 = xc;
            }
            if (lane < c) v0 = v0 - conj(d[tri(c, lane)]) * xc;
            if (lane + 32 < c) v1 = v1 - conj(d[tri(c, lane + 32)]) * xc;
        }
        if (lane < n) xs[lane] = v0;
        if (lane + 32 < n) xs[lane + 32] = v1;
    }
    __syncthreads();
    if (blockIdx.x == 0)
        for (int e = t; e < n; e += blockDim.x) x[base + e] = ccast<double>(xs[e]);
    // rows i in [32 blockIdx.x, +32): warp w sums the columns c in [8 w, 8 w + 8)
    // (coalesced along i), then warp 0 adds the eight partial sums
    __shared__ cpx<R> part[8][32];
    const int i = blockIdx.x * 32 + lane;
    cpx<R> s = {R(0), R(0)};
    if (i < base)
        for (int c = 8 * warp; c < 8 * warp + 8 && c < n; ++c)
            s = s + conj(L[(size_t)(base + c) * P + i]) * xs[c];
    part[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && i < base) {
        cpx<R> tot = part[0][lane];
        for (int w = 1; w < 8; ++w) tot = tot + part[w][lane];
        y[i] = y[i] - ccast<double>(tot);
    }
}

// x = 0, r = F, flags cleared; scal[1] = F.F (float64, one CTA).
__global__ void __launch_bounds__(1024) refine_init_kernel(const double* __restrict__ F_, int P,
                                                           double* __restrict__ x_,
                                                           double* __restrict__ r_,
                                                           double* __restrict__ scal) {
    __shared__ double red[32];
    const cpx<double>* F = (const cpx<double>*)F_;
    cpx<double>* x = (cpx<double>*)x_;
    cpx<double>* r = (cpx<double>*)r_;
    double s = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        x[k] = {0.0, 0.0};
        r[k] = F[k];
        s += abs2(F[k]);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 32; ++w) t += red[w];
        scal[1] = t;
        scal[2] = t > 0.0 ? 0.0 : 1.0;  // F = 0: x = 0 is exact
        scal[3] = 0.0;
        scal[4] = t;
        scal[8] = t;
    }
}

// r = F - S (x + d), one warp per row; per-CTA partial sums of |r|^2.
__global__ void __launch_bounds__(256) refine_resid_kernel(const double* __restrict__ S_, int P,
                                                           const double* __restrict__ F_,
                                                           const double* __restrict__ x_,
                                                           const double* __restrict__ d_,
                                                           double* __restrict__ r_,
                                                           double* __restrict__ part,
                                                           const double* __restrict__ skip) {
    if (*skip != 0.0) return;
    __shared__ double red[8];
    const cpx<double>* S = (const cpx<double>*)S_;
    const cpx<double>* x = (const cpx<double>*)x_;
    const cpx<double>* d = (const cpx<double>*)d_;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double acc = 0.0;
    for (int row = blockIdx.x * 8 + warp; row < P; row += gridDim.x * 8) {
        const cpx<double>* Sr = S + (size_t)row * P;
        cpx<double> s = {0.0, 0.0};
        for (int l = lane; l < P; l += 32) s = s + Sr[l] * (x[l] + d[l]);
        s = warp_sum(s);
        if (lane == 0) {
            const cpx<double> rv = ((const cpx<double>*)F_)[row] - s;
            ((cpx<double>*)r_)[row] = rv;
            acc += abs2(rv);
        }
    }
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}

// x += d; |r|^2 from the partial sums in a fixed order; stop on
// convergence or stagnation.
__global__ void __launch_bounds__(1024) refine_check_kernel(int P, double* __restrict__ x_,
                                                            const double* __restrict__ d_,
                                                            const double* __restrict__ part,
                                                            int npart, double tol,
                                                            double* __restrict__ scal) {
    if (scal[2] != 0.0) return;
    cpx<double>* x = (cpx<double>*)x_;
    const cpx<double>* d = (const cpx<double>*)d_;
    for (int k = threadIdx.x; k < P; k += blockDim.x) x[k] = x[k] + d[k];
    if (threadIdx.x == 0) {
        double rr = 0.0;
        for (int b = 0; b < npart; ++b) rr += part[b];
        const double prev = scal[8];
        scal[3] += 1.0;
        scal[4] = rr;
        scal[8] = rr;
        if (!(rr > tol * tol * scal[1]) || rr > 0.25 * prev) scal[2] = 1.0;
    }
}

template <typename R>
cr_status factor_t(cr_ctx* c) {
    const int P = c->P, nb = (P + NB - 1) / NB;
    cpx<R>* L = (cpx<R>*)c->Lf;
    const size_t n = (size_t)P * P;
    CR_LAUNCH(c, CR_K_OTHER,
              chol_copy_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->S, P, L));
    for (int J = 0; J < nb; ++J) {
        CR_LAUNCH(c, CR_KERNEL_CHOL, potrf_kernel<R><<<1, 256, 0, c->stream>>>(L, P, J, c->d_status));
        const int rows = P - (J + 1) * NB;
        if (rows <= 0) break;
        const int g = min((rows + 7) / 8, 4 * c->n_sm);
        CR_LAUNCH(c, CR_KERNEL_CHOL, trsm_kernel<R><<<g, 256, 0, c->stream>>>(L, P, J));
        const int T = nb - J - 1;
        CR_LAUNCH(c, CR_KERNEL_CHOL,
                  syrk_kernel<R><<<(unsigned)((long long)T * (T + 1) / 2), 256, 0, c->stream>>>(L, P, J));
    }
    return cr_check_launch(c, "blocked Cholesky");
}

template <typename R>
cr_status refine_t(cr_ctx* c, const double* F, int maxit) {
    const int P = c->P, nb = (P + NB - 1) / NB;
    const cpx<R>* L = (const cpx<R>*)c->Lf;
    double* x = c->cg;
    double* r = c->cg + 2 * (size_t)P;
    double* y = c->cg + 4 * (size_t)P;
    double* d = c->cg + 6 * (size_t)P;
    const double* done = c->scal + 2;
    CR_LAUNCH(c, CR_K_OTHER, refine_init_kernel<<<1, 1024, 0, c->stream>>>(F, P, x, r, c->scal));
    for (int it = 0; it < maxit; ++it) {
        for (int J = 0; J < nb; ++J) {
            const int rows = P - (J + 1) * NB;
            const int g = rows > 0 ? (rows + 31) / 32 : 1;
            CR_LAUNCH(c, CR_KERNEL_TRSV,
                      trsv_fwd_kernel<R><<<g, 256, 0, c->stream>>>(L, P, J, r, y, done));
        }
        for (int J = nb - 1; J >= 0; --J) {
            const int rows = J * NB;
            const int g = rows > 0 ? (rows + 31) / 32 : 1;
            CR_LAUNCH(c, CR_KERNEL_TRSV,
                      trsv_bwd_kernel<R><<<g, 256, 0, c->stream>>>(L, P, J, y, d, done));
        }
        CR_LAUNCH(c, CR_K_OTHER, refine_resid_kernel<<<RES_GRID, 256, 0, c->stream>>>(
                                     c->S, P, F, x, d, r, c->cgpart, done));
        CR_LAUNCH(c, CR_K_OTHER, refine_check_kernel<<<1, 1024, 0, c->stream>>>(
                                     P, x, d, c->cgpart, RES_GRID, REFINE_TOL, c->scal));
    }
    return cr_check_launch(c, "refined solve");
}

}  // namespace

bool chol_blocked(const cr_ctx* c) {
    return (c->flags & CR_CTX_EXPLICIT_S) && (c->prec != CR_FP64 || c->P > CHOL_SMALL_P);
}

size_t chol_factor_bytes(const cr_ctx* c) { return (size_t)c->P * c->P * 2 * rsize(c); }

size_t chol_cgpart_len() { return RES_GRID; }

cr_status chol_factor(cr_ctx* c) {
    return c->prec == CR_FP64 ? factor_t<double>(c) : factor_t<float>(c);
}

cr_status chol_refine_solve(cr_ctx* c, const double* F, int maxit) {
    if (maxit > REFINE_MAXIT) maxit = REFINE_MAXIT;
    if (maxit < 1) maxit = 1;
    return c->prec == CR_FP64 ? refine_t<double>(c, F, maxit) : refine_t<float>(c, F, maxit);
}
