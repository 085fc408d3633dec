// Chebyshev moment correction and the Krylov projection (Secs. IV, V).
//
// cheb_gram builds sigma_nm = <t_n|t_m> and H_nm = <t_n|H'|t_m> from the
// per-sample columns B_n(s) = t_n(s)/psi(s), (H' t_n)(s)/psi(s).
// cheb_krylov then works in float64: a complex Hermitian n x n matrix
// A = Ar + i Ai is handled through its real symmetric embedding
// [[Ar, -Ai], [Ai, Ar]] (every eigenvalue twice, eigenvector pairs
// [ur; ui], [-ui; ur]), diagonalised by cyclic Jacobi rotations applied to
// n disjoint pairs at a time (round-robin ordering), one launch per round on
// many CTAs; the moment recursion runs on one CTA.
#include "common.cuh"

// ------------------------------------------------------------------ Gram

template <typename R>
__global__ void gram_kernel(const cpx<R>* __restrict__ Bm, const cpx<R>* __restrict__ HBm, int Nm,
                            int B, int ld, double* __restrict__ G_, double* __restrict__ H_) {
    __shared__ cpx<R> tn[16][17], tm[16][17], th[16][17];
    const int n = blockIdx.y * 16 + threadIdx.y, m = blockIdx.x * 16 + threadIdx.x;
    cpx<double> g = {0.0, 0.0}, h = {0.0, 0.0};
    for (int s0 = 0; s0 < B; s0 += 16) {
        const int nn = blockIdx.y * 16 + threadIdx.y, s = s0 + threadIdx.x;
        tn[threadIdx.y][threadIdx.x] = (nn < Nm && s < B) ? Bm[(size_t)nn * ld + s] : cpx<R>{R(0), R(0)};
        const int mm = blockIdx.x * 16 + threadIdx.y;
        tm[threadIdx.y][threadIdx.x] = (mm < Nm && s < B) ? Bm[(size_t)mm * ld + s] : cpx<R>{R(0), R(0)};
        th[threadIdx.y][threadIdx.x] =
            (HBm && mm < Nm && s < B) ? HBm[(size_t)mm * ld + s] : cpx<R>{R(0), R(0)};
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            cpx<R> a = tn[threadIdx.y][q];
            g = g + ccast<double>(cmulc(a, tm[threadIdx.x][q]));
            h = h + ccast<double>(cmulc(a, th[threadIdx.x][q]));
        }
        __syncthreads();
    }
    if (n < Nm && m < Nm) {
        ((cpx<double>*)G_)[(size_t)n * Nm + m] = (1.0 / B) * g;
        if (H_) ((cpx<double>*)H_)[(size_t)n * Nm + m] = (1.0 / B) * h;
    }
}

__global__ void hermitise_kernel(double* __restrict__ H_, int Nm) {
    cpx<double>* H = (cpx<double>*)H_;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Nm * Nm) return;
    int n = idx / Nm, m = idx % Nm;
    if (m < n) return;
    cpx<double> a = H[(size_t)n * Nm + m], b = H[(size_t)m * Nm + n];
    cpx<double> v = 0.5 * (a + conj(b));
    H[(size_t)n * Nm + m] = v;
    H[(size_t)m * Nm + n] = conj(v);
}

extern "C" cr_status cheb_gram(cr_ctx* ctx, const void* Bmat, const void* HBmat, int Nm, int B,
                               int ld, double* G_out, double* H_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(Nm >= 1 && B >= 1 && ld >= B, "cheb_gram: bad sizes");
    CR_CHECK_ARG(Bmat && G_out && ((HBmat && H_out) || (!HBmat && !H_out)),
                 "cheb_gram: null array (HBmat and H_out are both given or both NULL)");
    if (ctx->prec == CR_MIXED) return launch_gram_tc(ctx, Bmat, HBmat, Nm, B, ld, G_out, H_out);
    dim3 g((Nm + 15) / 16, (Nm + 15) / 16);
    if (ctx->prec == CR_FP64)
        CR_LAUNCH(ctx, CR_K_OTHER, gram_kernel<double><<<g, dim3(16, 16), 0, ctx->stream>>>(
            (const cpx<double>*)Bmat, (const cpx<double>*)HBmat, Nm, B, ld, G_out, H_out));
    else
        CR_LAUNCH(ctx, CR_K_OTHER, gram_kernel<float><<<g, dim3(16, 16), 0, ctx->stream>>>(
            (const cpx<float>*)Bmat, (const cpx<float>*)HBmat, Nm, B, ld, G_out, H_out));
    if (H_out)
        CR_LAUNCH(ctx, CR_K_OTHER, hermitise_kernel<<<(Nm * Nm + 255) / 256, 256, 0, ctx->stream>>>(H_out, Nm));
    return cr_check_launch(ctx, "cheb_gram");
}

// ------------------------------------------------------------- Jacobi
//
// Cyclic Jacobi on many CTAs.  Each sweep has m - 1 rounds (round-robin
// pairing of the m indices: position 0 fixed, the others rotating); a round
// applies its m/2 disjoint rotations at once, A' = J^T A J and V' = V J, out
// of place (ping-pong buffers), one launch per round.  Every CTA computes
// the rotation angles of the pairs its 32 x 32 output tile touches from the
// round's input, so no launch waits on another.  Between sweeps the
// off-diagonal norm is reduced (fixed order) and, once it is below
// JAC_TOL times the diagonal, a device flag makes every later launch return
// at once; `res` records which buffer holds the latest A and V.

namespace {

constexpr int JAC_MAX_SWEEPS = 30;
constexpr double JAC_TOL = 1e-24;  // off^2 <= JAC_TOL diag^2 (relative 1e-12)
constexpr int NORM_GRID = 128;

// Element of the round-robin schedule: position 0 is fixed, the others
// rotate by one place per round.
__device__ __forceinline__ int rr_elem(int pos, int round, int m) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (m - 1)) + 1;
}
// Position of index idx in round `round` (inverse of rr_elem).
__device__ __forceinline__ int rr_pos(int idx, int round, int m) {
    return idx == 0 ? 0 : ((idx - 1 - round) % (m - 1) + (m - 1)) % (m - 1) + 1;
}

struct JacBufs {
    double* A[2];
    double* V[2];
    int* res;   // index of the buffers holding the latest A, V
    int* flag;  // converged
};

__global__ void jac_init_kernel(JacBufs J, int m) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) {
        *J.res = 0;
        *J.flag = 0;
    }
    if (idx < (size_t)m * m) J.V[0][idx] = (idx / m == idx % m) ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(256) jac_round_kernel(JacBufs J, int m, int round, int in) {
    if (*J.flag) return;
    __shared__ double ang_c[64], ang_s[64];
    __shared__ int partner[64], role[64];
    const double* A = J.A[in];
    const double* V = J.V[in];
    double* Ao = J.A[in ^ 1];
    double* Vo = J.V[in ^ 1];
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, t = threadIdx.x;
    if (t < 64) {
        const int idx = (t < 32 ? i0 : j0) + (t & 31);
        double c = 1.0, sn = 0.0;
        int pt = idx, rl = 0;
        if (idx < m) {
            const int pos = rr_pos(idx, round, m);
            const int k = pos < m / 2 ? pos : m - 1 - pos;
            const int p = rr_elem(k, round, m), q = rr_elem(m - 1 - k, round, m);
            const double apq = A[(size_t)p * m + q];
            if (apq != 0.0) {
                const double tau = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
                const double tt = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                c = 1.0 / sqrt(1.0 + tt * tt);
                sn = tt * c;
            }
            pt = idx == p ? q : p;
            rl = idx == p ? 0 : 1;
        }
        ang_c[t] = c;
        ang_s[t] = sn;
        partner[t] = pt;
        role[t] = rl;
    }
    __syncthreads();
    for (int e = t; e < 1024; e += blockDim.x) {
        const int li = e >> 5, lj = e & 31, i = i0 + li, j = j0 + lj;
        if (i >= m || j >= m) continue;
        const double ci = ang_c[li], si = ang_s[li], cj = ang_c[32 + lj], sj = ang_s[32 + lj];
        const int ip = partner[li], jp = partner[32 + lj];
        // column step (pair of j) on rows i and i', then the row step (pair of i)
        const double sgj = role[32 + lj] ? sj : -sj, sgi = role[li] ? si : -si;
        const double bij = cj * A[(size_t)i * m + j] + sgj * A[(size_t)i * m + jp];
        const double bpj = cj * A[(size_t)ip * m + j] + sgj * A[(size_t)ip * m + jp];
        Ao[(size_t)i * m + j] = ci * bij + sgi * bpj;
        Vo[(size_t)i * m + j] = cj * V[(size_t)i * m + j] + sgj * V[(size_t)i * m + jp];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && t == 0) *J.res = in ^ 1;
}

// Per-CTA shares of the squared off-diagonal and diagonal sums of A[res].
__global__ void __launch_bounds__(256) jac_norm_kernel(JacBufs J, int m, double* __restrict__ part) {
    if (*J.flag) return;
    __shared__ double r1[8], r2[8];
    const double* A = J.A[*J.res];
    double off = 0.0, dia = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)m * m;
         e += (size_t)gridDim.x * blockDim.x) {
        const double v = A[e] * A[e];
        if (e / m == e % m) dia += v;
        else off += v;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = off;
        r2[threadIdx.x >> 5] = dia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += r1[w];
            b += r2[w];
        }
        part[blockIdx.x] = a;
        part[NORM_GRID + blockIdx.x] = b;
    }
}

__global__ void jac_flag_kernel(JacBufs J, const double* __restrict__ part) {
    if (*J.flag) return;
    double off = 0.0, dia = 0.0;
    for (int b = 0; b < NORM_GRID; ++b) {
        off += part[b];
        dia += part[NORM_GRID + b];
    }
    if (!(off > JAC_TOL * dia)) *J.flag = 1;
}

// Diagonalise the symmetric m x m matrix in J.A[0] (m even); eigenvalues on
// the diagonal of J.A[*res], eigenvectors in the columns of J.V[*res].
void jacobi_launch(cr_ctx* c, JacBufs J, int m, double* part) {
    const size_t mm = (size_t)m * m;
    CR_LAUNCH(c, CR_K_OTHER, jac_init_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, c->stream>>>(J, m));
    const dim3 g((m + 31) / 32, (m + 31) / 32);
    int in = 0;
    for (int sweep = 0; sweep < JAC_MAX_SWEEPS; ++sweep) {
        CR_LAUNCH(c, CR_K_OTHER, jac_norm_kernel<<<NORM_GRID, 256, 0, c->stream>>>(J, m, part));
        CR_LAUNCH(c, CR_K_OTHER, jac_flag_kernel<<<1, 1, 0, c->stream>>>(J, part));
        for (int round = 0; round < m - 1; ++round) {
            CR_LAUNCH(c, CR_K_OTHER, jac_round_kernel<<<g, 256, 0, c->stream>>>(J, m, round, in));
            in ^= 1;
        }
    }
}

// Real symmetric embedding [[Ar, -Ai], [Ai, Ar]] of a complex Hermitian n x n
// matrix (every eigenvalue twice, eigenvector pairs [ur; ui], [-ui; ur]).
__global__ void kry_embed_kernel(const double* __restrict__ A_, int n, double* __restrict__ E) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int m = 2 * n, i = e / n, j = e % n;
    const cpx<double> a = ((const cpx<double>*)A_)[e];
    E[(size_t)i * m + j] = a.x;
    E[(size_t)(i + n) * m + j + n] = a.x;
    E[(size_t)(i + n) * m + j] = a.y;
    E[(size_t)i * m + j + n] = -a.y;
}

// Eigenvalues of the embedded G, the kept index list (relative cutoff; an
// odd count drops the smallest, the copy a cutoff split by rounding) and
// the rank r (even).  One thread.
__global__ void kry_keep_kernel(JacBufs J, int m, double cutoff, double* __restrict__ d,
                                int* __restrict__ keep, int* __restrict__ rank) {
    const double* E = J.A[*J.res];
    double dm = 0.0;
    for (int k = 0; k < m; ++k) {
        d[k] = E[(size_t)k * m + k];
        dm = d[k] > dm ? d[k] : dm;
    }
    int r = 0;
    for (int k = 0; k < m; ++k)
        if (d[k] > cutoff * dm) keep[r++] = k;
    if (r & 1) {
        int lo = 0;
        for (int q = 1; q < r; ++q)
            if (d[keep[q]] < d[keep[lo]]) lo = q;
        for (int q = lo; q < r - 1; ++q) keep[q] = keep[q + 1];
        --r;
    }
    *rank = r;
}

// Y[i][j] = sum_kept V[i][k] V[j][k] / d[k], i < m, j < n: the pseudo-inverse
// of the embedded G, first n columns (G^+ = Y[0:n] + i Y[n:2n]).
__global__ void kry_pinv_kernel(JacBufs J, int m, const double* __restrict__ d,
                                const int* __restrict__ keep, const int* __restrict__ rank,
                                double* __restrict__ Y) {
    const int n = m / 2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * n) return;
    const double* V = J.V[*J.res];
    const int i = e / n, j = e % n, r = *rank;
    double s = 0.0;
    for (int q = 0; q < r; ++q) {
        const int k = keep[q];
        s += V[(size_t)i * m + k] * V[(size_t)j * m + k] / d[k];
    }
    Y[e] = s;
}

// X[i][q] = V[i][keep q] / sqrt(d) for q < r, 0 for r <= q < m (padding).
__global__ void kry_x_kernel(JacBufs J, int m, const double* __restrict__ d,
                             const int* __restrict__ keep, const int* __restrict__ rank,
                             double* __restrict__ X) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int i = e / m, q = e % m, r = *rank;
    const double* V = J.V[*J.res];
    X[e] = q < r ? V[(size_t)i * m + keep[q]] / sqrt(d[keep[q]]) : 0.0;
}

// C = A^T B or A B (m x m, row-major), one output per thread (float64).
template <bool TRANS_A>
__global__ void kry_gemm_kernel(const double* __restrict__ A, const double* __restrict__ B, int m,
                                double* __restrict__ C) {
    __shared__ double as[16][17], bs[16][17];
    const int i = blockIdx.y * 16 + threadIdx.y, j = blockIdx.x * 16 + threadIdx.x;
    double s = 0.0;
    for (int l0 = 0; l0 < m; l0 += 16) {
        const int la = l0 + threadIdx.x, lb = l0 + threadIdx.y;
        const int ia = blockIdx.y * 16 + threadIdx.y;
        as[threadIdx.y][threadIdx.x] =
            (ia < m && la < m) ? (TRANS_A ? A[(size_t)la * m + ia] : A[(size_t)ia * m + la]) : 0.0;
        bs[threadIdx.y][threadIdx.x] = (lb < m && j < m) ? B[(size_t)lb * m + j] : 0.0;
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) s += as[threadIdx.y][q] * bs[q][threadIdx.x];
        __syncthreads();
    }
    if (i < m && j < m) C[(size_t)i * m + j] = s;
}

// out = (C + C^T) / 2 into the Jacobi input buffer; g0 = X^T [Re G e0; Im G e0].
__global__ void kry_sym_kernel(const double* __restrict__ C, int m, double* __restrict__ out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m * m) return;
    const int a = e / m, b = e % m;
    out[e] = 0.5 * (C[e] + C[(size_t)b * m + a]);
}

__global__ void kry_g0_kernel(const double* __restrict__ G_, const double* __restrict__ X, int m,
                              double* __restrict__ g0) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    const int n = m / 2;
    const cpx<double>* G = (const cpx<double>*)G_;
    double s = 0.0;
    for (int l = 0; l < n; ++l) {
        const cpx<double> gl = G[(size_t)l * n];
        s += X[(size_t)l * m + q] * gl.x + X[(size_t)(l + n) * m + q] * gl.y;
    }
    g0[q] = s;
}

// Moment correction (one CTA): c_0 = e_0, c_1 = G^+ H c_0,
// c_{k+1} = G^+ (2 H c_k - G c_{k-1}); mu'_k = (G c_k)_0.
__global__ void __launch_bounds__(1024) kry_moments_kernel(const double* __restrict__ G_,
                                                           const double* __restrict__ H_, int n,
                                                           const double* __restrict__ Y, int n_out,
                                                           double* __restrict__ vec,
                                                           double* __restrict__ mu_out) {
    const cpx<double>* G = (const cpx<double>*)G_;
    const cpx<double>* H = (const cpx<double>*)H_;
    cpx<double>* c0 = (cpx<double>*)vec;
    cpx<double>* c1 = c0 + n;
    cpx<double>* t1 = c1 + n;
    cpx<double>* t2 = t1 + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        c0[i] = {i == 0 ? 1.0 : 0.0, 0.0};
        c1[i] = {0.0, 0.0};
    }
    __syncthreads();
    for (int k = 0; k < n_out; ++k) {
        if (threadIdx.x == 0) {
            cpx<double> s = {0.0, 0.0};
            for (int l = 0; l < n; ++l) s = s + G[l] * c0[l];
            mu_out[2 * k] = s.x;
            mu_out[2 * k + 1] = s.y;
        }
        if (k == n_out - 1) break;
        // t1 = (k == 0 ? H c0 : 2 H c0 - G c1)   (c1 holds c_{k-1})
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            cpx<double> s = {0.0, 0.0}, gsum = {0.0, 0.0};
            for (int l = 0; l < n; ++l) {
                s = s + H[(size_t)i * n + l] * c0[l];
                gsum = gsum + G[(size_t)i * n + l] * c1[l];
            }
            t1[i] = k == 0 ? s : (2.0 * s - gsum);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            cpx<double> s = {0.0, 0.0};
            for (int l = 0; l < n; ++l) {
                const cpx<double> gp = {Y[(size_t)i * n + l], Y[(size_t)(i + n) * n + l]};
                s = s + gp * t1[l];
            }
            t2[i] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            c1[i] = c0[i];
            c0[i] = t2[i];
        }
        __syncthreads();
    }
}

// Poles and weights from the diagonalised projection (one CTA): eigenvalue
// k = E[k][k] for k < r, weight (V[:, k] . g0)^2; sorted, and the doubled
// eigenvalues of the embedding merged in pairs.
__global__ void __launch_bounds__(1024) kry_final_kernel(JacBufs J, int m,
                                                         const double* __restrict__ g0,
                                                         const int* __restrict__ rank,
                                                         double* __restrict__ d,
                                                         double* __restrict__ wk,
                                                         double* __restrict__ poles,
                                                         double* __restrict__ weights,
                                                         int32_t* __restrict__ rank_out) {
    const double* E = J.A[*J.res];
    const double* V = J.V[*J.res];
    const int r = *rank, n = m / 2;
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < r; ++q) s += V[(size_t)q * m + k] * g0[q];
        wk[k] = s * s;
        d[k] = E[(size_t)k * m + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < r; ++i) {
            const double dv = d[i], wv = wk[i];
            int j = i - 1;
            while (j >= 0 && d[j] > dv) {
                d[j + 1] = d[j];
                wk[j + 1] = wk[j];
                --j;
            }
            d[j + 1] = dv;
            wk[j + 1] = wv;
        }
        for (int k = 0; k < n; ++k) {
            if (2 * k + 1 < r) {
                poles[k] = 0.5 * (d[2 * k] + d[2 * k + 1]);
                weights[k] = wk[2 * k] + wk[2 * k + 1];
            } else {
                poles[k] = 0.0;
                weights[k] = 0.0;
            }
        }
        if (rank_out) *rank_out = r / 2;
    }
}

}  // namespace

extern "C" cr_status cheb_krylov(cr_ctx* ctx, const double* G, const double* H, int Nm,
                                 double cutoff, int n_out, double* mu_corr_out, double* poles_out,
                                 double* weights_out, int32_t* rank_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(Nm >= 1 && Nm <= 512, "cheb_krylov: Nm=%d outside [1, 512]", Nm);
    CR_CHECK_ARG(n_out >= 1, "cheb_krylov: n_out < 1");
    CR_CHECK_ARG(G && H && mu_corr_out && poles_out && weights_out, "cheb_krylov: null array");
    const int n = Nm, m = 2 * Nm;
    const size_t mm = (size_t)m * m;
    // workspace (doubles): A0, A1, V0, V1, X, C [m*m]; Y [m*n]; d, wk, g0 [m];
    // 4 complex vectors [n]; norm shares [2 NORM_GRID]; ints: keep [m], rank, res, flag
    const size_t need = 6 * mm + (size_t)m * n + 3 * (size_t)m + 8 * (size_t)n +
                        2 * NORM_GRID + ((size_t)m + 3 + 1) / 2 + 1;
    if (ctx->kry_len < need) {
        // first use at this size: the only allocation outside cr_create
        if (ctx->kry) cudaFree(ctx->kry);
        ctx->kry = nullptr;
        ctx->kry_len = 0;
        if (cudaMalloc((void**)&ctx->kry, need * sizeof(double)) != cudaSuccess)
            return cr_fail(ctx, CR_ENOMEM, "cheb_krylov: workspace");
        ctx->kry_len = need;
    }
    double* w = ctx->kry;
    JacBufs J;
    J.A[0] = w;
    J.A[1] = w + mm;
    J.V[0] = w + 2 * mm;
    J.V[1] = w + 3 * mm;
    double* X = w + 4 * mm;
    double* C = w + 5 * mm;
    double* Y = w + 6 * mm;
    double* d = Y + (size_t)m * n;
    double* wk = d + m;
    double* g0 = wk + m;
    double* vec = g0 + m;
    double* part = vec + 8 * (size_t)n;
    int* keep = (int*)(part + 2 * NORM_GRID);
    int* rank = keep + m;
    J.res = rank + 1;
    J.flag = rank + 2;
    const unsigned gm = (unsigned)((mm + 255) / 256);
    const unsigned gn = (unsigned)(((size_t)n * n + 255) / 256);
    const dim3 g16((m + 15) / 16, (m + 15) / 16);
    cudaStream_t st = ctx->stream;
    // 1. G through its embedding: eigenvalues, kept rank, pseudo-inverse
    cudaError_t e = cudaMemsetAsync(J.A[0], 0, mm * sizeof(double), st);
    if (e != cudaSuccess) return cr_fail(ctx, CR_ECUDA, "cheb_krylov: %s", cudaGetErrorString(e));
    CR_LAUNCH(ctx, CR_K_OTHER, kry_embed_kernel<<<gn, 256, 0, st>>>(G, n, J.A[0]));
    jacobi_launch(ctx, J, m, part);
    CR_LAUNCH(ctx, CR_K_OTHER, kry_keep_kernel<<<1, 1, 0, st>>>(J, m, cutoff, d, keep, rank));
    CR_LAUNCH(ctx, CR_K_OTHER,
              kry_pinv_kernel<<<(unsigned)(((size_t)m * n + 255) / 256), 256, 0, st>>>(J, m, d, keep, rank, Y));
    // 2. corrected moments
    CR_LAUNCH(ctx, CR_K_OTHER, kry_moments_kernel<<<1, 1024, 0, st>>>(G, H, n, Y, n_out, vec, mu_corr_out));
    // 3. projected eigenproblem: X = V_kept d^-1/2 (zero-padded to m columns),
    //    Hx = X^T Hemb X, diagonalised by the same Jacobi (padding stays zero)
    CR_LAUNCH(ctx, CR_K_OTHER, kry_x_kernel<<<gm, 256, 0, st>>>(J, m, d, keep, rank, X));
    CR_LAUNCH(ctx, CR_K_OTHER, kry_g0_kernel<<<(m + 255) / 256, 256, 0, st>>>(G, X, m, g0));
    e = cudaMemsetAsync(C, 0, mm * sizeof(double), st);
    if (e != cudaSuccess) return cr_fail(ctx, CR_ECUDA, "cheb_krylov: %s", cudaGetErrorString(e));
    CR_LAUNCH(ctx, CR_K_OTHER, kry_embed_kernel<<<gn, 256, 0, st>>>(H, n, C));
    CR_LAUNCH(ctx, CR_K_OTHER, kry_gemm_kernel<false><<<g16, dim3(16, 16), 0, st>>>(C, X, m, J.A[1]));
    CR_LAUNCH(ctx, CR_K_OTHER, kry_gemm_kernel<true><<<g16, dim3(16, 16), 0, st>>>(X, J.A[1], m, C));
    CR_LAUNCH(ctx, CR_K_OTHER, kry_sym_kernel<<<gm, 256, 0, st>>>(C, m, J.A[0]));
    jacobi_launch(ctx, J, m, part);
    CR_LAUNCH(ctx, CR_K_OTHER,
              kry_final_kernel<<<1, 1024, 0, st>>>(J, m, g0, rank, d, wk, poles_out, weights_out, rank_out));
    return cr_check_launch(ctx, "cheb_krylov");
}
