// The RBM ansatz of Sec. I: theta = b + sigma W, log psi, bond-ratio tables,
// and the explicit log-derivatives of Sec. III.
#include "common.cuh"

// ------------------------------------------------------------------ tables
//
// Exchanging the antiparallel spins of bond (i, i') with s = sigma_i changes
// theta_m by -s D_m, D_m = 2 (W_im - W_i'm), so
//   cosh(theta_m - s D_m) / cosh(theta_m) = cosh D_m - s tanh(theta_m) sinh D_m
// and the visible factor by exp(-s 2 (a_i - a_i')).  The tables hold D, cosh D,
// sinh D per (bond, hidden unit), padded to Mp columns with the neutral
// values (0, 1, 0), and exp(-/+ 2 (a_i - a_i')) per bond.
template <typename R>
__global__ void tables_kernel(const cpx<R>* __restrict__ prm, const int2* __restrict__ bonds, int N,
                              int M, int Mp, int Nb, cpx<R>* D, cpx<R>* Ch, cpx<R>* Sh, cpx<R>* ChT,
                              cpx<R>* ShT, cpx<R>* ea) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Nb * Mp) return;
    int b = idx / Mp, m = idx % Mp;
    int2 bd = bonds[b];
    cpx<R> d = {R(0), R(0)}, ch = {R(1), R(0)}, sh = {R(0), R(0)};
    if (m < M) {
        const cpx<R>* W = prm + N + M;
        cpx<R> wi = W[(size_t)bd.x * M + m], wj = W[(size_t)bd.y * M + m];
        d = R(2) * (wi - wj);
        ccoshsinh_(d, &ch, &sh);
    }
    D[idx] = d;
    Ch[idx] = ch;
    Sh[idx] = sh;
    ChT[(size_t)m * Nb + b] = ch;
    ShT[(size_t)m * Nb + b] = sh;
    if (m == 0) {
        cpx<R> da = R(2) * (prm[bd.x] - prm[bd.y]);
        ea[2 * b] = cexp_(-da);
        ea[2 * b + 1] = cexp_(da);
    }
}

template <typename R>
static cr_status build_tables_t(cr_ctx* c, const void* params, int slot) {
    const cr_tables& t = c->tab[slot];
    int n = c->Nb * c->Mp;
    CR_LAUNCH(c, CR_K_OTHER, tables_kernel<R><<<(n + 255) / 256, 256, 0, c->stream>>>(
        (const cpx<R>*)params, c->d_bonds, c->N, c->M, c->Mp, c->Nb, (cpx<R>*)t.D, (cpx<R>*)t.Ch,
        (cpx<R>*)t.Sh, (cpx<R>*)t.ChT, (cpx<R>*)t.ShT, (cpx<R>*)t.ea));
    return cr_check_launch(c, "tables_kernel");
}

cr_status build_tables(cr_ctx* c, const void* params, int slot) {
    return c->prec == CR_FP64 ? build_tables_t<double>(c, params, slot)
                              : build_tables_t<float>(c, params, slot);
}

// ------------------------------------------------------ theta and log psi
//
// One CTA of 128 threads takes WB walkers; thread t owns hidden units
// j = t + 128 k (k < JPT) for all WB walkers, so every W element loaded
// from L1/L2 feeds 2 WB FMAs (sigma = +-1 is exact in R).  Epilogue:
//   MODE_LOGPSI: theta_out = theta, out = a.sigma + sum_j log 2cosh theta_j
//   MODE_MATVEC: out = v_a.sigma + sum_j T_j (v_b + sigma V_W)_j, i.e. O v
//                with O_a = sigma, O_b = T, O_W = sigma (x) T (Sec. III).
enum { MODE_LOGPSI = 0, MODE_MATVEC = 1 };

template <typename R, int JPT, int WB, int MODE>
__global__ void __launch_bounds__(128) theta_kernel(const cpx<R>* __restrict__ prm,
                                                    const int8_t* __restrict__ spins, int B, int N,
                                                    int M, cpx<R>* __restrict__ theta_out,
                                                    cpx<R>* __restrict__ out,
                                                    const cpx<R>* __restrict__ T,
                                                    const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;  // converged CG: nothing left to do
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sg = (R*)smem_raw;                       // [N][WB]: the WB signs of site i together
    cpx<R>* red = (cpx<R>*)(sg + WB * N);       // [4][WB]
    const int w0 = blockIdx.x * WB;
    const int t = threadIdx.x;
    for (int e = t; e < WB * N; e += 128) {
        int w = e / N, i = e % N;
        sg[i * WB + w] = (w0 + w < B) ? R(spins[(size_t)(w0 + w) * N + i]) : R(0);
    }
    __syncthreads();
    const cpx<R>* a = prm;
    const cpx<R>* b = prm + N;
    const cpx<R>* W = prm + N + M;
    cpx<R> acc[WB][JPT];
#pragma unroll
    for (int k = 0; k < JPT; ++k) {
        int j = t + 128 * k;
        cpx<R> bj = j < M ? b[j] : cpx<R>{R(0), R(0)};
#pragma unroll
        for (int w = 0; w < WB; ++w) acc[w][k] = bj;
    }
    // W rows are loaded one step ahead so that their latency overlaps the FMAs
    cpx<R> wnext[JPT];
#pragma unroll
    for (int k = 0; k < JPT; ++k) {
        int j = t + 128 * k;
        wnext[k] = (j < M && N > 0) ? W[j] : cpx<R>{R(0), R(0)};
    }
    for (int i = 0; i < N; ++i) {
        cpx<R> wv[JPT];
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            wv[k] = wnext[k];
            int j = t + 128 * k;
            wnext[k] = (j < M && i + 1 < N) ? W[(size_t)(i + 1) * M + j] : cpx<R>{R(0), R(0)};
        }
        // WB signs in 16-byte shared loads
        R sv[WB];
#pragma unroll
        for (int w = 0; w < WB; w += 16 / sizeof(R)) {
            uint4 v = *reinterpret_cast<const uint4*>(sg + i * WB + w);
            memcpy(&sv[w], &v, 16);
        }
#pragma unroll
        for (int w = 0; w < WB; ++w) {
#pragma unroll
            for (int k = 0; k < JPT; ++k) {
                acc[w][k].x = fma(sv[w], wv[k].x, acc[w][k].x);
                acc[w][k].y = fma(sv[w], wv[k].y, acc[w][k].y);
            }
        }
    }
    cpx<R> part[WB];
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        part[w] = {R(0), R(0)};
        const bool live = w0 + w < B;
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            int j = t + 128 * k;
            if (j < M && live) {
                if (MODE == MODE_LOGPSI) {
                    if (theta_out) theta_out[(size_t)(w0 + w) * M + j] = acc[w][k];
                    part[w] = part[w] + clncosh2_(acc[w][k]);
                } else {
                    part[w] = part[w] + T[(size_t)(w0 + w) * M + j] * acc[w][k];
                }
            }
        }
        for (int i = t; i < N; i += 128) part[w] = part[w] + sg[i * WB + w] * a[i];
    }
    const int lane = t & 31, wid = t >> 5;
#pragma unroll
    for (int w = 0; w < WB; ++w) {
        cpx<R> v = warp_sum(part[w]);
        if (lane == 0) red[wid * WB + w] = v;
    }
    __syncthreads();
    if (t < WB && w0 + t < B) {
        cpx<R> s = red[t] + red[WB + t] + red[2 * WB + t] + red[3 * WB + t];
        out[w0 + t] = s;
    }
}

template <typename R, int MODE>
static cr_status launch_theta_t(cr_ctx* c, const void* params, const int8_t* spins, int B,
                                void* theta, void* out, const void* T, const double* skip) {
    if (B == 0) return CR_OK;
    const int jpt = (c->M + 127) / 128;
    const int N = c->N;
#define LAUNCH(JPT, WB)                                                                          \
    {                                                                                            \
        size_t sm = WB * N * sizeof(R) + 4 * WB * sizeof(cpx<R>);                                \
        CR_LAUNCH(c, (MODE == MODE_LOGPSI ? CR_KERNEL_THETA : CR_KERNEL_OV), theta_kernel<R, JPT, WB, MODE><<<(B + WB - 1) / WB, 128, sm, c->stream>>>(               \
            (const cpx<R>*)params, spins, B, N, c->M, (cpx<R>*)theta, (cpx<R>*)out,              \
            (const cpx<R>*)T, skip));                                                             \
    }
    if (jpt == 1) LAUNCH(1, 16)
    else if (jpt == 2) LAUNCH(2, 16)
    else if (jpt <= 4) LAUNCH(4, 8)
    else LAUNCH(8, 4)
#undef LAUNCH
    return cr_check_launch(c, "theta_kernel");
}

cr_status launch_logpsi(cr_ctx* c, const void* params, const int8_t* spins, int B, void* theta,
                        void* logpsi) {
    return c->prec == CR_FP64
               ? launch_theta_t<double, MODE_LOGPSI>(c, params, spins, B, theta, logpsi, nullptr,
                                                     nullptr)
               : launch_theta_t<float, MODE_LOGPSI>(c, params, spins, B, theta, logpsi, nullptr,
                                                    nullptr);
}

// u_s = sum_k O_k(s) v_k for the structured O of Sec. III.
cr_status launch_ov(cr_ctx* c, const void* v, const int8_t* spins, int B, const void* T, void* u,
                    const double* skip) {
    return c->prec == CR_FP64
               ? launch_theta_t<double, MODE_MATVEC>(c, v, spins, B, nullptr, u, T, skip)
               : launch_theta_t<float, MODE_MATVEC>(c, v, spins, B, nullptr, u, T, skip);
}

// ------------------------------------------------------------- logderiv

template <typename R>
__global__ void tanh_kernel(const cpx<R>* __restrict__ theta, size_t n, cpx<R>* __restrict__ out) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] = ctanh_(theta[idx]);
}

template <typename R>
__global__ void o_explicit_kernel(const int8_t* __restrict__ spins, const cpx<R>* __restrict__ theta,
                                  int B, int N, int M, int P, cpx<R>* __restrict__ O) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * P) return;
    int s = (int)(idx / P), k = (int)(idx % P);
    cpx<R> v;
    if (k < N) {
        v = {R(spins[(size_t)s * N + k]), R(0)};
    } else if (k < N + M) {
        v = ctanh_(theta[(size_t)s * M + (k - N)]);
    } else {
        int i = (k - N - M) / M, j = (k - N - M) % M;
        v = R(spins[(size_t)s * N + i]) * ctanh_(theta[(size_t)s * M + j]);
    }
    O[idx] = v;
}

template <typename R>
static cr_status logderiv_t(cr_ctx* ctx, const int8_t* spins, const void* theta, int B,
                            void* tanh_out, void* O_out) {
    if (tanh_out) {
        size_t n = (size_t)B * ctx->M;
        CR_LAUNCH(ctx, CR_K_OTHER, tanh_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            (const cpx<R>*)theta, n, (cpx<R>*)tanh_out));
    }
    if (O_out) {
        size_t n = (size_t)B * ctx->P;
        CR_LAUNCH(ctx, CR_K_OTHER, o_explicit_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
            spins, (const cpx<R>*)theta, B, ctx->N, ctx->M, ctx->P, (cpx<R>*)O_out));
    }
    return cr_check_launch(ctx, "logderiv");
}

cr_status logderiv_impl(cr_ctx* ctx, const int8_t* spins, const void* theta, int B, void* tanh_out,
                        void* O_out) {
    return ctx->prec == CR_FP64 ? logderiv_t<double>(ctx, spins, theta, B, tanh_out, O_out)
                                : logderiv_t<float>(ctx, spins, theta, B, tanh_out, O_out);
}

// --------------------------------------------------------------- C ABI

extern "C" cr_status rbm_logpsi(cr_ctx* ctx, const cr_state* st, const int8_t* spins, int B,
                                void* theta_out, void* logpsi_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(st && st->params, "rbm_logpsi: null state");
    CR_CHECK_ARG(B >= 0 && B <= ctx->max_walkers, "rbm_logpsi: B=%d outside [0, %d]", B,
                 ctx->max_walkers);
    if (B == 0) return CR_OK;
    CR_CHECK_ARG(spins && logpsi_out, "rbm_logpsi: null spins or output");
    return launch_logpsi(ctx, st->params, spins, B, theta_out, logpsi_out);
}

extern "C" cr_status logderiv(cr_ctx* ctx, const cr_state* st, const int8_t* spins,
                              const void* theta, int B, void* tanh_out, void* O_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(st && st->params, "logderiv: null state");
    CR_CHECK_ARG(B >= 0 && B <= ctx->max_walkers, "logderiv: B=%d outside [0, %d]", B,
                 ctx->max_walkers);
    if (B == 0) return CR_OK;
    CR_CHECK_ARG(spins && theta, "logderiv: null spins or theta");
    return logderiv_impl(ctx, spins, theta, B, tanh_out, O_out);
}

// ------------------------------------------------- start of projection step n
//
// The recursion of Sec. III fits RBM_n from a starting point the paper leaves
// open.  RBM_1 starts from psi with a_0 += i pi/2: e^{i pi sigma_0 / 2} =
// i sigma_0, so that RBM equals 2i S^z_0 psi exactly, a state with weight on
// H' S^z_q psi; RBM_n (n >= 2) starts from RBM_{n-1} (warm start).
template <typename R>
__global__ void init_params_kernel(const cpx<R>* __restrict__ src, int P, int shift_a0,
                                   cpx<R>* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    cpx<R> v = src[k];
    if (shift_a0 && k == 0) v.y += R(1.5707963267948966);  // + i pi/2
    out[k] = v;
}

extern "C" cr_status cheb_init_params(cr_ctx* ctx, int n, const void* psi, const void* prev,
                                      void* out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(n >= 1, "cheb_init_params: n must be >= 1");
    CR_CHECK_ARG(out && (n == 1 ? psi != nullptr : prev != nullptr),
                 "cheb_init_params: null parameter vector");
    const void* src = n == 1 ? psi : prev;
    const int P = ctx->P, g = (P + 255) / 256;
    if (ctx->prec == CR_FP64)
        CR_LAUNCH(ctx, CR_K_OTHER, init_params_kernel<double><<<g, 256, 0, ctx->stream>>>(
                                       (const cpx<double>*)src, P, n == 1, (cpx<double>*)out));
    else
        CR_LAUNCH(ctx, CR_K_OTHER, init_params_kernel<float><<<g, 256, 0, ctx->stream>>>(
                                       (const cpx<float>*)src, P, n == 1, (cpx<float>*)out));
    return cr_check_launch(ctx, "init_params_kernel");
}
