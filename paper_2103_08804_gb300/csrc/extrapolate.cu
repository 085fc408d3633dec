// Extrapolation of Chebyshev moments by linear prediction (Sec. VI).
//
// The paper notes that higher moments can be approximated from the known
// ones by extrapolation, citing the Chebyshev-MPS literature; it gives no
// algorithm.  This is linear prediction as applied to Chebyshev moments by
// Ganahl, Thunstroem, Verstraete, Held and Evertz, Phys. Rev. B 90, 045144
// (2014), with the growing-mode treatment of Barthel, Schollwoeck and White,
// Phys. Rev. B 79, 245101 (2009):
//   1. a_1..a_p minimise sum_{n=n0}^{N-1} |mu_n + sum_i a_i mu_{n-i}|^2:
//      normal equations (R + delta I) a = -r, delta = reg * max_i R_ii,
//      solved by Cholesky;
//   2. the roots z_k of z^p + a_1 z^{p-1} + ... + a_p, found together by the
//      Aberth-Ehrlich iteration (O. Aberth, Math. Comp. 27 (1973) 339), and
//      the amplitudes c_k of mu_n = sum_k c_k z_k^n fitted to the last p
//      known moments (Vandermonde system, LU with partial pivoting);
//   3. roots outside the unit circle are moved onto it, w_k = z_k / |z_k|;
//   4. mu_{N-p+m} = sum_k c_k w_k^m for m >= p.
// One CTA per sequence, float64 throughout; every loop has a fixed bound.
#include "common.cuh"

namespace {

constexpr int LP_THREADS = 256;
constexpr int LP_MAX_ORDER = 512;
constexpr int ABERTH_MAX_IT = 500;

using zd = cpx<double>;

CR_D double cabs1(zd a) { return fabs(a.x) + fabs(a.y); }

// z^m by binary powering
CR_D zd zpow(zd z, int m) {
    zd r = {1.0, 0.0};
    while (m > 0) {
        if (m & 1) r = r * z;
        z = z * z;
        m >>= 1;
    }
    return r;
}

// Block-wide maximum of v (every thread gets it).
CR_D double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

// Block-wide argmax of (v, i) with the smallest i among equal maxima.
CR_D int block_argmax(double v, int i, double* red, int* redi) {
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (v2 > v || (v2 == v && i2 < i)) {
            v = v2;
            i = i2;
        }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = v;
        redi[threadIdx.x >> 5] = i;
    }
    __syncthreads();
    double bv = red[0];
    int bi = redi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (red[w] > bv || (red[w] == bv && redi[w] < bi)) {
            bv = red[w];
            bi = redi[w];
        }
    __syncthreads();
    return bi;
}

struct LpArgs {
    const zd* mu;      // [n_seq][N]
    int N, p, n0;
    double reg;
    int n_out;
    zd* mu_out;        // [n_seq][n_out]
    zd* roots_out;     // [n_seq][p] or null
    int* info;         // [n_seq] or null
    zd* work;          // [n_seq][2 p p]
    int* status;
};

__global__ void __launch_bounds__(LP_THREADS) lp_kernel(const LpArgs A) {
    __shared__ zd sa[LP_MAX_ORDER];   // right-hand sides, then a; later b, then c
    __shared__ zd sz[LP_MAX_ORDER];   // roots
    __shared__ zd sz2[LP_MAX_ORDER];  // next iterate of the roots
    __shared__ zd sq[LP_MAX_ORDER];   // polynomial coefficients a_1..a_p
    __shared__ double red[32];
    __shared__ int redi[32];
    __shared__ int flag, done;
    const int tid = threadIdx.x, nt = blockDim.x, s = blockIdx.x;
    const int N = A.N, p = A.p, n0 = A.n0;
    const zd* mu = A.mu + (size_t)s * N;
    zd* out = A.mu_out + (size_t)s * A.n_out;
    zd* R = A.work + (size_t)s * 2 * p * p;
    zd* V = R + (size_t)p * p;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (tid == 0) flag = 0;

    // 1. normal equations over the targets n = n0 .. N-1 (lags i + 1, j + 1)
    for (int e = tid; e < p * p; e += nt) {
        const int i = e / p, j = e % p;
        zd acc = {0.0, 0.0};
        for (int n = n0; n < N; ++n) acc = acc + cmulc(mu[n - 1 - i], mu[n - 1 - j]);
        R[e] = acc;
    }
    for (int i = tid; i < p; i += nt) {
        zd acc = {0.0, 0.0};
        for (int n = n0; n < N; ++n) acc = acc + cmulc(mu[n - 1 - i], mu[n]);
        sa[i] = -acc;
    }
    __syncthreads();
    double dmax = 0.0;
    for (int i = tid; i < p; i += nt) dmax = fmax(dmax, R[(size_t)i * p + i].x);
    dmax = block_max(dmax, red);
    for (int i = tid; i < p; i += nt) R[(size_t)i * p + i].x += A.reg * dmax;
    __syncthreads();

    // Cholesky R = L L^dag (lower triangle, in place)
    for (int k = 0; k < p; ++k) {
        if (tid == 0) {
            const double d = R[(size_t)k * p + k].x;
            if (!(d > 0.0)) flag = 1;
            else R[(size_t)k * p + k] = {sqrt(d), 0.0};
        }
        __syncthreads();
        if (flag) break;
        const double il = 1.0 / R[(size_t)k * p + k].x;
        for (int i = k + 1 + tid; i < p; i += nt) R[(size_t)i * p + k] = il * R[(size_t)i * p + k];
        __syncthreads();
        const int w = p - k - 1;
        for (int e = tid; e < w * w; e += nt) {
            const int i = k + 1 + e / w, j = k + 1 + e % w;
            if (j <= i) R[(size_t)i * p + j] = R[(size_t)i * p + j] - R[(size_t)i * p + k] * conj(R[(size_t)j * p + k]);
        }
        __syncthreads();
    }
    if (!flag) {
        // L y = -r, then L^dag a = y
        for (int k = 0; k < p; ++k) {
            if (tid == 0) sa[k] = (1.0 / R[(size_t)k * p + k].x) * sa[k];
            __syncthreads();
            for (int i = k + 1 + tid; i < p; i += nt) sa[i] = sa[i] - R[(size_t)i * p + k] * sa[k];
            __syncthreads();
        }
        for (int k = p - 1; k >= 0; --k) {
            if (tid == 0) sa[k] = (1.0 / R[(size_t)k * p + k].x) * sa[k];
            __syncthreads();
            for (int i = tid; i < k; i += nt) sa[i] = sa[i] - conj(R[(size_t)k * p + i]) * sa[k];
            __syncthreads();
        }
    }

    // 2a. roots of z^p + a_1 z^{p-1} + ... + a_p (Aberth-Ehrlich, all roots
    // updated together from the previous iterate)
    int iters = -1;
    if (!flag) {
        for (int i = tid; i < p; i += nt) sq[i] = sa[i];
        const double ap = sqrt(abs2(sa[p - 1]));
        const double rho = ap > 0.0 ? fmin(fmax(pow(ap, 1.0 / p), 1e-3), 1e3) : 1.0;
        for (int k = tid; k < p; k += nt) {
            double sn, cs;
            sincos(6.283185307179586 * k / p + 0.7, &sn, &cs);
            sz[k] = {rho * cs, rho * sn};
        }
        __syncthreads();
        for (int it = 0; it < ABERTH_MAX_IT; ++it) {
            if (tid == 0) done = 1;
            __syncthreads();
            for (int k = tid; k < p; k += nt) {
                const zd z = sz[k];
                zd P = {1.0, 0.0}, dP = {0.0, 0.0};
                for (int i = 0; i < p; ++i) {
                    dP = dP * z + P;
                    P = P * z + sq[i];
                }
                zd S = {0.0, 0.0};
                for (int j = 0; j < p; ++j)
                    if (j != k) {
                        const zd d = z - sz[j];
                        if (abs2(d) > 0.0) S = S + cdiv(zd{1.0, 0.0}, d);
                    }
                zd delta = {0.0, 0.0};
                if (abs2(P) > 0.0) {
                    const zd Nr = abs2(dP) > 0.0 ? cdiv(P, dP) : zd{1e-3, 1e-3};
                    const zd den = zd{1.0, 0.0} - Nr * S;
                    delta = abs2(den) > 0.0 ? cdiv(Nr, den) : Nr;
                }
                sz2[k] = z - delta;
                if (sqrt(abs2(delta)) > 1e-14 * fmax(1.0, sqrt(abs2(z)))) done = 0;
            }
            __syncthreads();
            for (int k = tid; k < p; k += nt) sz[k] = sz2[k];
            __syncthreads();
            const int converged = done;
            __syncthreads();  // every thread has read done before it is reset
            if (converged) {
                iters = it + 1;
                break;
            }
        }
    }

    // 2b. amplitudes: sum_k c_k z_k^m = mu_{N-p+m}, m < p (V[m][k] = z_k^m)
    if (!flag) {
        for (int e = tid; e < p * p; e += nt) V[e] = zpow(sz[e % p], e / p);
        for (int m = tid; m < p; m += nt) sa[m] = mu[N - p + m];
        __syncthreads();
        for (int k = 0; k < p; ++k) {
            double bv = -1.0;
            int bi = k;
            for (int i = k + tid; i < p; i += nt) {
                const double v = cabs1(V[(size_t)i * p + k]);
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
            const int piv = block_argmax(bv, bi, red, redi);
            if (tid == 0 && !(cabs1(V[(size_t)piv * p + k]) > 0.0)) flag = 1;
            __syncthreads();
            if (flag) break;
            if (piv != k) {
                for (int j = tid; j < p; j += nt) {
                    const zd t = V[(size_t)k * p + j];
                    V[(size_t)k * p + j] = V[(size_t)piv * p + j];
                    V[(size_t)piv * p + j] = t;
                }
                if (tid == 0) {
                    const zd t = sa[k];
                    sa[k] = sa[piv];
                    sa[piv] = t;
                }
            }
            __syncthreads();
            const zd piv_v = V[(size_t)k * p + k];
            for (int i = k + 1 + tid; i < p; i += nt) {
                const zd l = cdiv(V[(size_t)i * p + k], piv_v);
                V[(size_t)i * p + k] = l;
                sa[i] = sa[i] - l * sa[k];
            }
            __syncthreads();
            const int w = p - k - 1;
            for (int e = tid; e < w * w; e += nt) {
                const int i = k + 1 + e / w, j = k + 1 + e % w;
                V[(size_t)i * p + j] = V[(size_t)i * p + j] - V[(size_t)i * p + k] * V[(size_t)k * p + j];
            }
            __syncthreads();
        }
        if (!flag)
            for (int k = p - 1; k >= 0; --k) {
                if (tid == 0) sa[k] = cdiv(sa[k], V[(size_t)k * p + k]);
                __syncthreads();
                for (int i = tid; i < k; i += nt) sa[i] = sa[i] - V[(size_t)i * p + k] * sa[k];
                __syncthreads();
            }
    }

    // 3, 4. stabilised roots (in sz2) and the prediction
    for (int k = tid; k < p; k += nt) {
        const zd z = sz[k];
        const double az = sqrt(abs2(z));
        sz2[k] = az > 1.0 ? (1.0 / az) * z : z;
        if (A.roots_out) A.roots_out[(size_t)s * p + k] = flag ? zd{nan, nan} : z;
    }
    __syncthreads();
    for (int n = tid; n < N; n += nt) out[n] = mu[n];
    for (int t = tid; t < A.n_out - N; t += nt) {
        zd acc = {0.0, 0.0};
        if (flag) {
            acc = {nan, nan};
        } else {
            const double m = (double)(p + t);
            for (int k = 0; k < p; ++k) {
                const zd w = sz2[k];
                const double lw = 0.5 * log(abs2(w)), ph = atan2(w.y, w.x);
                double sn, cs;
                sincos(m * ph, &sn, &cs);
                const double mag = exp(m * lw);
                acc = acc + sa[k] * zd{mag * cs, mag * sn};
            }
        }
        out[N + t] = acc;
    }
    if (tid == 0) {
        if (A.info) A.info[s] = flag ? -2 : iters;
        if (flag) set_status(A.status, CR_ESINGULAR);
    }
}

}  // namespace

extern "C" cr_status cheb_extrapolate(cr_ctx* ctx, const double* mu, int n_seq, int n_known,
                                      int order, int n0, double reg, int n_out, double* mu_out,
                                      double* roots_out, int* info_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(mu && mu_out, "cheb_extrapolate: null moments");
    CR_CHECK_ARG(n_seq >= 1 && order >= 1 && order <= LP_MAX_ORDER,
                 "cheb_extrapolate: need n_seq >= 1 and 1 <= order <= %d", LP_MAX_ORDER);
    CR_CHECK_ARG(order <= n0 && n0 < n_known && n_known <= n_out,
                 "cheb_extrapolate: need order <= n0 < n_known <= n_out");
    CR_CHECK_ARG(reg >= 0.0, "cheb_extrapolate: reg < 0");
    const size_t need = (size_t)n_seq * 2 * order * order * sizeof(zd);
    cr_status st = cr_grow(ctx, (void**)&ctx->lp_work, &ctx->lp_work_cap, need, "cheb_extrapolate");
    if (st != CR_OK) return st;
    LpArgs a;
    a.mu = (const zd*)mu;
    a.N = n_known;
    a.p = order;
    a.n0 = n0;
    a.reg = reg;
    a.n_out = n_out;
    a.mu_out = (zd*)mu_out;
    a.roots_out = (zd*)roots_out;
    a.info = info_out;
    a.work = (zd*)ctx->lp_work;
    a.status = ctx->d_status;
    CR_LAUNCH(ctx, CR_K_OTHER, lp_kernel<<<n_seq, LP_THREADS, 0, ctx->stream>>>(a));
    return cr_check_launch(ctx, "lp_kernel");
}
