// Symmetry projection of the local Chebyshev sequence onto every momentum
// of the L x L square lattice (Appendix A).
//
// For each sample s, the 4 N transformed configurations
//   s'(x) = s(R^r x + m + d_r),  r = 0..3, m in the L x L translations,
//   d_r = (0,0), (1,0), (1,1), (0,1)  (the translation paired with R^r in P^(R)),
// R (x, y) = (-y, x) mod L, are built once; for each stored state t_n the
// log-amplitudes at all of them come from the theta kernel in one launch,
// then
//   A_m(s)  = (1/4) sum_r t_n(s'_{m,r}) / psi(s),
//   B~_nk(s) = L^-1 sum_m e^{-i 2 pi k.m / L} A_m(s),
// for all momenta k = (k1, k2) (index k1 + L k2), in the context precision.
#include "common.cuh"

namespace {

__device__ __forceinline__ void rot(int& x, int& y, int r, int L) {
    for (int q = 0; q < r; ++q) {
        const int nx = (L - y) % L;
        y = x;
        x = nx;
    }
}

__global__ void sym_permute_kernel(const int8_t* __restrict__ spins, int B, int L,
                                   int8_t* __restrict__ out) {
    const int N = L * L;
    const size_t total = (size_t)4 * N * B * N;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int x = (int)(idx % N);
    const size_t rest = idx / N;
    const int s = (int)(rest % B);
    const int g = (int)(rest / B), r = g / N, m = g % N;
    const int dx = (r == 1 || r == 2) ? 1 : 0, dy = (r == 2 || r == 3) ? 1 : 0;
    int rx = x % L, ry = x / L;
    rot(rx, ry, r, L);
    const int src = (rx + m % L + dx) % L + L * ((ry + m / L + dy) % L);
    out[idx] = spins[(size_t)s * N + src];
}

// A[m][s] = (1/4) sum_r exp(lp[(r N + m) B + s] - lp_ref[s])
template <typename R>
__global__ void sym_rot_kernel(const cpx<R>* __restrict__ lp, const cpx<R>* __restrict__ lp_ref,
                               int N, int B, cpx<R>* __restrict__ A) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * B) return;
    const int m = (int)(idx / B), s = (int)(idx % B);
    const cpx<R> ref = lp_ref[s];
    cpx<R> acc = {R(0), R(0)};
#pragma unroll
    for (int r = 0; r < 4; ++r) acc = acc + cexp_(lp[((size_t)r * N + m) * B + s] - ref);
    A[idx] = R(0.25) * acc;
}

// Bt[(k Nm + n) B + s] = L^-1 sum_m e^{-i 2 pi (k1 m1 + k2 m2) / L} A[m][s]
template <typename R>
__global__ void sym_dft_kernel(const cpx<R>* __restrict__ A, int L, int B, int n, int Nm,
                               cpx<R>* __restrict__ Bt) {
    extern __shared__ __align__(16) unsigned char smem[];
    cpx<R>* ph = (cpx<R>*)smem;  // [L] e^{-i 2 pi j / L}
    const int N = L * L;
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        R sn, cs;
        m_sincos(R(2.0 * 3.14159265358979323846 * j / L), &sn, &cs);
        ph[j] = {cs, -sn};
    }
    __syncthreads();
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * B) return;
    const int k = (int)(idx / B), s = (int)(idx % B), k1 = k % L, k2 = k / L;
    cpx<R> acc = {R(0), R(0)};
    for (int m = 0; m < N; ++m) {
        const int e = (k1 * (m % L) + k2 * (m / L)) % L;
        acc = acc + ph[e] * A[(size_t)m * B + s];
    }
    Bt[((size_t)k * Nm + n) * B + s] = (R(1) / R(L)) * acc;
}

size_t ws_layout(const cr_ctx* c, int B, size_t* off_lp, size_t* off_A) {
    const size_t N = c->N, cs = 2 * (size_t)rsize(c);
    const size_t sp = ((4 * N * B * N + 255) / 256) * 256;
    *off_lp = sp;
    *off_A = sp + ((4 * N * B * cs + 255) / 256) * 256;
    return *off_A + N * B * cs;
}

template <typename R>
cr_status btilde_t(cr_ctx* c, const cr_state* states, int Nm, const int8_t* spins,
                   const void* lp_ref, int B, unsigned char* ws, void* Bt) {
    const int L = c->Lx, N = c->N;
    size_t off_lp, off_A;
    ws_layout(c, B, &off_lp, &off_A);
    int8_t* sp = (int8_t*)ws;
    cpx<R>* lp = (cpx<R>*)(ws + off_lp);
    cpx<R>* A = (cpx<R>*)(ws + off_A);
    const size_t np = (size_t)4 * N * B * N;
    CR_LAUNCH(c, CR_K_OTHER, sym_permute_kernel<<<(unsigned)((np + 255) / 256), 256, 0, c->stream>>>(spins, B, L, sp));
    const size_t nb = (size_t)N * B;
    for (int n = 0; n < Nm; ++n) {
        cr_status s = launch_logpsi(c, states[n].params, sp, 4 * N * B, nullptr, lp);
        if (s != CR_OK) return s;
        CR_LAUNCH(c, CR_K_OTHER, sym_rot_kernel<R><<<(unsigned)((nb + 255) / 256), 256, 0, c->stream>>>(
                                     lp, (const cpx<R>*)lp_ref, N, B, A));
        CR_LAUNCH(c, CR_K_OTHER,
                  sym_dft_kernel<R><<<(unsigned)((nb + 255) / 256), 256, L * sizeof(cpx<R>), c->stream>>>(
                      A, L, B, n, Nm, (cpx<R>*)Bt));
    }
    return cr_check_launch(c, "sym_btilde");
}

}  // namespace

extern "C" size_t sym_workspace_bytes(const cr_ctx* ctx, int B) {
    if (!ctx || B < 1) return 0;
    size_t a, b;
    return ws_layout(ctx, B, &a, &b);
}

extern "C" cr_status sym_btilde(cr_ctx* ctx, const cr_state* states, int Nm, const int8_t* spins,
                                const void* logpsi_ref, int B, void* workspace,
                                size_t workspace_bytes, void* Bt_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(ctx->Ly == ctx->Lx, "sym_btilde: needs a square L x L lattice");
    CR_CHECK_ARG(Nm >= 1 && B >= 1, "sym_btilde: Nm and B must be >= 1");
    CR_CHECK_ARG((size_t)4 * ctx->N * B <= (size_t)0x7fffffff, "sym_btilde: 4 N B too large");
    CR_CHECK_ARG(states && spins && logpsi_ref && workspace && Bt_out, "sym_btilde: null array");
    CR_CHECK_ARG(workspace_bytes >= sym_workspace_bytes(ctx, B),
                 "sym_btilde: workspace of %zu bytes, need %zu", workspace_bytes,
                 sym_workspace_bytes(ctx, B));
    for (int n = 0; n < Nm; ++n)
        CR_CHECK_ARG(states[n].params && !states[n].probe,
                     "sym_btilde: state %d: plain RBM states only (no probe factor)", n);
    return ctx->prec == CR_FP64
               ? btilde_t<double>(ctx, states, Nm, spins, logpsi_ref, B, (unsigned char*)workspace, Bt_out)
               : btilde_t<float>(ctx, states, Nm, spins, logpsi_ref, B, (unsigned char*)workspace, Bt_out);
}
