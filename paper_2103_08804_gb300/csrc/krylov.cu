// Chebyshev moment correction and the Krylov projection (Secs. IV, V).
//
// cheb_gram builds sigma_nm = <t_n|t_m> and H_nm = <t_n|H'|t_m> from the
// per-sample columns B_n(s) = t_n(s)/psi(s), (H' t_n)(s)/psi(s).
// cheb_krylov then works in float64 on one CTA: a complex Hermitian n x n
// matrix A = Ar + i Ai is handled through its real symmetric embedding
// [[Ar, -Ai], [Ai, Ar]] (every eigenvalue twice, eigenvector pairs
// [ur; ui], [-ui; ur]), diagonalised by cyclic Jacobi rotations applied to
// n disjoint pairs at a time (round-robin ordering).
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
        th[threadIdx.y][threadIdx.x] = (mm < Nm && s < B) ? HBm[(size_t)mm * ld + s] : cpx<R>{R(0), R(0)};
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
        ((cpx<double>*)H_)[(size_t)n * Nm + m] = (1.0 / B) * h;
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
    CR_CHECK_ARG(Bmat && HBmat && G_out && H_out, "cheb_gram: null array");
    dim3 g((Nm + 15) / 16, (Nm + 15) / 16);
    if (ctx->prec == CR_FP64)
        CR_LAUNCH(ctx, CR_K_OTHER, gram_kernel<double><<<g, dim3(16, 16), 0, ctx->stream>>>(
            (const cpx<double>*)Bmat, (const cpx<double>*)HBmat, Nm, B, ld, G_out, H_out));
    else
        CR_LAUNCH(ctx, CR_K_OTHER, gram_kernel<float><<<g, dim3(16, 16), 0, ctx->stream>>>(
            (const cpx<float>*)Bmat, (const cpx<float>*)HBmat, Nm, B, ld, G_out, H_out));
    CR_LAUNCH(ctx, CR_K_OTHER, hermitise_kernel<<<(Nm * Nm + 255) / 256, 256, 0, ctx->stream>>>(H_out, Nm));
    return cr_check_launch(ctx, "cheb_gram");
}

// ------------------------------------------------------------- Jacobi

// Element of the round-robin schedule: position 0 is fixed, the others
// rotate by one place per round.
__device__ __forceinline__ int rr_elem(int pos, int round, int m) {
    return pos == 0 ? 0 : ((pos - 1 + round) % (m - 1)) + 1;
}

// Diagonalise the symmetric m x m matrix A (row-major, in place; m even)
// and accumulate the rotations into V (V = eigenvectors as columns).
// cs: scratch [m] (cos, sin per pair).  Whole CTA participates.
__device__ void jacobi_sym(double* A, double* V, int m, double* cs, int max_sweeps) {
    __shared__ double red[32];
    __shared__ int stop;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) V[e] = (e / m == e % m) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            double v = A[e] * A[e];
            if (e / m == e % m) dia += v;
            else off += v;
        }
        __syncthreads();
        off = warp_sum(off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = off;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            red[0] = t;
        }
        __syncthreads();
        off = red[0];
        __syncthreads();
        dia = warp_sum(dia);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dia;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
            stop = !(off > 1e-30 * t) ? 1 : 0;
        }
        __syncthreads();
        if (stop) break;
        for (int round = 0; round < m - 1; ++round) {
            // rotation angles for the m/2 disjoint pairs of this round
            for (int k = threadIdx.x; k < m / 2; k += blockDim.x) {
                int p = rr_elem(k, round, m), q = rr_elem(m - 1 - k, round, m);
                double apq = A[(size_t)p * m + q], c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    double tau = (A[(size_t)q * m + q] - A[(size_t)p * m + p]) / (2.0 * apq);
                    double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + t * t);
                    s = t * c;
                }
                cs[2 * k] = c;
                cs[2 * k + 1] = s;
            }
            __syncthreads();
            // A <- A J (columns p, q) and V <- V J
            for (int e = threadIdx.x; e < (m / 2) * m; e += blockDim.x) {
                int k = e / m, r = e % m;
                int p = rr_elem(k, round, m), q = rr_elem(m - 1 - k, round, m);
                double c = cs[2 * k], s = cs[2 * k + 1];
                double ap = A[(size_t)r * m + p], aq = A[(size_t)r * m + q];
                A[(size_t)r * m + p] = c * ap - s * aq;
                A[(size_t)r * m + q] = s * ap + c * aq;
                double vp = V[(size_t)r * m + p], vq = V[(size_t)r * m + q];
                V[(size_t)r * m + p] = c * vp - s * vq;
                V[(size_t)r * m + q] = s * vp + c * vq;
            }
            __syncthreads();
            // A <- J^T A (rows p, q)
            for (int e = threadIdx.x; e < (m / 2) * m; e += blockDim.x) {
                int k = e / m, r = e % m;
                int p = rr_elem(k, round, m), q = rr_elem(m - 1 - k, round, m);
                double c = cs[2 * k], s = cs[2 * k + 1];
                double ap = A[(size_t)p * m + r], aq = A[(size_t)q * m + r];
                A[(size_t)p * m + r] = c * ap - s * aq;
                A[(size_t)q * m + r] = s * ap + c * aq;
            }
            __syncthreads();
        }
    }
    __syncthreads();
}

// Real symmetric embedding of a complex Hermitian n x n matrix.
__device__ void embed(const cpx<double>* A, int n, double* E) {
    const int m = 2 * n;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;
        cpx<double> a = A[e];
        E[(size_t)i * m + j] = a.x;
        E[(size_t)(i + n) * m + j + n] = a.x;
        E[(size_t)(i + n) * m + j] = a.y;
        E[(size_t)i * m + j + n] = -a.y;
    }
}

// Workspace layout (doubles): E [m*m], V [m*m], X [m*m], Y [m*m], small vectors.
__global__ void __launch_bounds__(1024) krylov_kernel(const double* __restrict__ G_,
                                                      const double* __restrict__ H_, int n,
                                                      double cutoff, int n_out, double* __restrict__ ws,
                                                      double* __restrict__ mu_out,
                                                      double* __restrict__ poles,
                                                      double* __restrict__ weights,
                                                      int32_t* __restrict__ rank_out) {
    const cpx<double>* G = (const cpx<double>*)G_;
    const cpx<double>* H = (const cpx<double>*)H_;
    const int m = 2 * n;
    const size_t mm = (size_t)m * m;
    double* E = ws;
    double* V = ws + mm;
    double* X = ws + 2 * mm;
    double* Y = ws + 3 * mm;
    double* d = ws + 4 * mm;       // [m] eigenvalues of the embedded G
    double* cs = d + m;            // [m]
    double* w = cs + m;            // [m]
    cpx<double>* c0 = (cpx<double>*)(w + m);   // [n] x 4 complex vectors
    cpx<double>* c1 = c0 + n;
    cpx<double>* t1 = c1 + n;
    cpx<double>* t2 = t1 + n;
    __shared__ int s_keep[1024];
    __shared__ int s_rank;

    // 1. G = U L U^dag through the embedding
    embed(G, n, E);
    __syncthreads();
    jacobi_sym(E, V, m, cs, 60);
    for (int k = threadIdx.x; k < m; k += blockDim.x) d[k] = E[(size_t)k * m + k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double dm = 0.0;
        for (int k = 0; k < m; ++k) dm = d[k] > dm ? d[k] : dm;
        int r = 0;
        for (int k = 0; k < m; ++k)
            if (d[k] > cutoff * dm) s_keep[r++] = k;
        if (r & 1) {
            // the embedding doubles every eigenvalue; a cutoff that splits a
            // pair by rounding drops the smaller copy
            int lo = 0;
            for (int q = 1; q < r; ++q)
                if (d[s_keep[q]] < d[s_keep[lo]]) lo = q;
            for (int q = lo; q < r - 1; ++q) s_keep[q] = s_keep[q + 1];
            --r;
        }
        s_rank = r;
    }
    __syncthreads();
    const int r = s_rank;
    // 2. pseudo-inverse G^+ in the embedding: Y = sum_kept v v^T / d
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        double s = 0.0;
        for (int q = 0; q < r; ++q) {
            int k = s_keep[q];
            s += V[(size_t)i * m + k] * V[(size_t)j * m + k] / d[k];
        }
        Y[e] = s;
    }
    __syncthreads();
    // 3. moment correction: c_0 = e_0, c_1 = G^+ H c_0, c_{k+1} = G^+ (2 H c_k - G c_{k-1});
    //    mu'_k = (G c_k)_0.  G^+ = Y[0:n,0:n] + i Y[n:2n,0:n].
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        c0[i] = {i == 0 ? 1.0 : 0.0, 0.0};
        c1[i] = {0.0, 0.0};
    }
    __syncthreads();
    for (int k = 0; k < n_out; ++k) {
        // mu'_k = sum_l G_0l c_k[l]
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
                cpx<double> gp = {Y[(size_t)i * m + l], Y[(size_t)(i + n) * m + l]};
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
    __syncthreads();
    // 4. projected eigenproblem: Xh = Vk diag(d^-1/2) (m x r), Hx = Xh^T Hemb Xh
    embed(H, n, E);
    __syncthreads();
    // X[i][q] = V[i][keep q] / sqrt(d)
    for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
        int i = e / r, q = e % r, k = s_keep[q];
        X[(size_t)i * r + q] = V[(size_t)i * m + k] / sqrt(d[k]);
    }
    __syncthreads();
    // Y = Hemb X  (m x r)
    for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
        int i = e / r, q = e % r;
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += E[(size_t)i * m + l] * X[(size_t)l * r + q];
        Y[e] = s;
    }
    __syncthreads();
    // E = X^T Y (r x r), symmetrised
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        int a = e / r, b = e % r;
        double s = 0.0;
        for (int l = 0; l < m; ++l) s += X[(size_t)l * r + a] * Y[(size_t)l * r + b];
        V[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
        int a = e / r, b = e % r;
        E[e] = 0.5 * (V[e] + V[(size_t)b * r + a]);
    }
    __syncthreads();
    // g0 = X^T (G e_0 embedded) = X^T [Re G[:,0]; Im G[:,0]]
    for (int q = threadIdx.x; q < r; q += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) {
            cpx<double> gl = G[(size_t)l * n];
            s += X[(size_t)l * r + q] * gl.x + X[(size_t)(l + n) * r + q] * gl.y;
        }
        w[q] = s;
    }
    __syncthreads();
    jacobi_sym(E, V, r, cs, 60);   // r is even: kept eigenvalues come in pairs
    // eigenvalue k: E[k][k]; weight: (V[:,k] . g0)^2
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < r; ++q) s += V[(size_t)q * r + k] * w[q];
        cs[k] = s * s;
        d[k] = E[(size_t)k * r + k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // sort ascending (insertion sort, r <= 1024), then merge the pairs
        for (int i = 1; i < r; ++i) {
            double dv = d[i], wv = cs[i];
            int j = i - 1;
            while (j >= 0 && d[j] > dv) {
                d[j + 1] = d[j];
                cs[j + 1] = cs[j];
                --j;
            }
            d[j + 1] = dv;
            cs[j + 1] = wv;
        }
        for (int k = 0; k < n; ++k) {
            if (2 * k + 1 < r) {
                poles[k] = 0.5 * (d[2 * k] + d[2 * k + 1]);
                weights[k] = cs[2 * k] + cs[2 * k + 1];
            } else {
                poles[k] = 0.0;
                weights[k] = 0.0;
            }
        }
        if (rank_out) *rank_out = r / 2;
    }
}

extern "C" cr_status cheb_krylov(cr_ctx* ctx, const double* G, const double* H, int Nm,
                                 double cutoff, int n_out, double* mu_corr_out, double* poles_out,
                                 double* weights_out, int32_t* rank_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(Nm >= 1 && Nm <= 512, "cheb_krylov: Nm=%d outside [1, 512]", Nm);
    CR_CHECK_ARG(n_out >= 1, "cheb_krylov: n_out < 1");
    CR_CHECK_ARG(G && H && mu_corr_out && poles_out && weights_out, "cheb_krylov: null array");
    const size_t m = 2 * (size_t)Nm;
    const size_t need = 4 * m * m + 3 * m + 8 * (size_t)Nm;
    if (ctx->kry_len < need) {
        // first use at this size: the only allocation outside cr_create
        if (ctx->kry) cudaFree(ctx->kry);
        ctx->kry = nullptr;
        ctx->kry_len = 0;
        if (cudaMalloc((void**)&ctx->kry, need * sizeof(double)) != cudaSuccess)
            return cr_fail(ctx, CR_ENOMEM, "cheb_krylov: workspace");
        ctx->kry_len = need;
    }
    CR_LAUNCH(ctx, CR_K_OTHER, krylov_kernel<<<1, 1024, 0, ctx->stream>>>(G, H, Nm, cutoff, n_out, ctx->kry, mu_corr_out,
                                               poles_out, weights_out, rank_out));
    return cr_check_launch(ctx, "krylov_kernel");
}
