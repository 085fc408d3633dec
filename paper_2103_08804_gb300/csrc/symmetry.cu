// Symmetry projection of the local Chebyshev sequence onto every momentum
// of the L x L square lattice (Appendix A).
//
// Each term T_{d_r} R^r of the rotation projector P^(R), d_r = (0,0), (1,0),
// (1,1), (0,1), is the r-fold quarter turn about the probe site: the paper's
// R turns the lattice about a plaquette centre and the paired translation
// returns the S^z operator to the origin, which is what makes P^(R) leave the
// exact t_n00 unchanged.  So for each sample s the 4 N transformed
// configurations
//   s'_{m,r}(x) = s(Q^r x + m),  r = 0..3, m in the L x L translations,
// with Q (x, y) = (-y, x) mod L the quarter turn about site (0, 0), are built
// once; for each stored state t_n the
// log-amplitudes at all of them come from the theta kernel in one launch,
// then
//   A_m(s)  = (1/4) sum_r t_n(s'_{m,r}) / psi(s),
//   B~_nk(s) = L^-1 sum_m e^{-i 2 pi k.m / L} A_m(s),
// for all momenta k = (k1, k2) (index k1 + L k2), in the context precision.
//
// The projected Hamiltonian follows the same route: H' commutes with every
// lattice map, so H' t~_nk = L P_k^(T) P^(R) H' t_n00 and
//   HB~_nk(s) = <s|H'|t~_nk> / psi(s)
// is the same rotation average and Fourier sum taken over
// (H' t_n)(s') / psi(s) at each transformed configuration.  That value is
// formed without dividing by t_n(s'): the transformed configurations are not
// samples of |t_n|^2 and can sit next to a node of t_n (cosh theta_m ~ 0),
// where the ratio tables of the target kernel (tanh theta) lose all
// precision in float32.
#include "common.cuh"

namespace {

__device__ __forceinline__ void rot(int& x, int& y, int r, int L) {
    for (int q = 0; q < r; ++q) {
        const int nx = (L - y) % L;
        y = x;
        x = nx;
    }
}

// out[((r N + m) B + s) N + x] = s(Q^r x + m)
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
    int rx = x % L, ry = x / L;
    rot(rx, ry, r, L);
    const int src = (rx + m % L) % L + L * ((ry + m / L) % L);
    out[idx] = spins[(size_t)s * N + src];
}

// A[m][s] = (1/4) sum_r exp(lp[(r N + m) B + s] - lp_ref[s]), and when hb
// is given HA[m][s] = (1/4) sum_r hb[(r N + m) B + s]
template <typename R>
__global__ void sym_rot_kernel(const cpx<R>* __restrict__ lp, const cpx<R>* __restrict__ lp_ref,
                               const cpx<R>* __restrict__ hb, int N, int B,
                               cpx<R>* __restrict__ A, cpx<R>* __restrict__ HA) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)N * B) return;
    const int m = (int)(idx / B), s = (int)(idx % B);
    const cpx<R> ref = lp_ref[s];
    cpx<R> acc = {R(0), R(0)}, hacc = {R(0), R(0)};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const size_t g = ((size_t)r * N + m) * B + s;
        acc = acc + cexp_(lp[g] - ref);
        if (hb) hacc = hacc + hb[g];
    }
    A[idx] = R(0.25) * acc;
    if (hb) HA[idx] = R(0.25) * hacc;
}

// hb[w] = (H' t_n)(s'_w) / psi(s), w = g B + s over the nc transformed
// configurations (Sec. V bonds).  With x_m = Re theta_m(s'),
// C_m = cosh(theta_m) e^{-|x_m|} and S_m = sinh(theta_m) e^{-|x_m|} (both of
// modulus <= 1),
//   t_n(s'^{ij}) / psi(s) = e^{Lam} ea_b prod_m (C_m cosh D_bm - s_i S_m sinh D_bm),
//   Lam = a.s' + M log 2 + sum_m |x_m| - log psi(s),
// from cosh(theta - s D) = cosh theta cosh D - s sinh theta sinh D and the
// bond tables D_bm, ea_b of t_n; the products are rescaled by a power of
// two every 16 factors and Lam, the diagonal part and the sums are formed in
// float64.
//
// One lane per configuration: the 32 lanes of a warp walk the same bonds
// and hidden units in step, so every table read is one broadcast for the
// whole warp, and a lane keeps GB independent bond products in registers
// (GB bonds per pass over the hidden units).  Every bond is evaluated and the
// parallel ones are dropped from the sum, which costs twice the arithmetic
// of the antiparallel bonds alone but no divergence.  theta of the warp's 32
// configurations is staged through shared memory MC hidden units at a time
// (coalesced reads), and C_m, S_m are formed again on every pass.
constexpr int SYM_MC = 8;

template <typename R>
CR_HD constexpr int sym_gb() { return sizeof(R) == 4 ? 16 : 8; }

template <typename R>
__global__ void __launch_bounds__(128) sym_hprime_kernel(
    const int8_t* __restrict__ sp, const cpx<R>* __restrict__ theta, const cpx<R>* __restrict__ lp,
    const cpx<R>* __restrict__ lp_ref, const cpx<R>* __restrict__ a_vis,
    const cpx<R>* __restrict__ ChT, const cpx<R>* __restrict__ ShT, const cpx<R>* __restrict__ ea,
    const int2* __restrict__ bonds_g, int nc, int B, int N, int M, int Mp, int Nb, double J,
    double E0, double a, double Wp, cpx<R>* __restrict__ hb) {
    constexpr int GB = sym_gb<R>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Nq = (N + 3) & ~3;
    int2* bonds = (int2*)smem_raw;                                   // [Nb]
    cpx<R>* thall = (cpx<R>*)(bonds + Nb + (Nb & 1));                // [4][SYM_MC][32]
    int8_t* sgall = (int8_t*)(thall + 4 * 32 * SYM_MC);              // [128][Nq]
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int wb = blockIdx.x * 128;                                 // first configuration of the block
    const int w = wb + t;
    const bool valid = w < nc;
    for (int e = t; e < Nb; e += 128) bonds[e] = bonds_g[e];
    const int nblk = nc - wb < 128 ? nc - wb : 128;
    for (int e = t; e < nblk * N; e += 128) sgall[(e / N) * Nq + e % N] = sp[(size_t)wb * N + e];
    __syncthreads();
    const int8_t* sg = sgall + t * Nq;
    cpx<R>* th = thall + wid * 32 * SYM_MC;
    cpx<double> as = {0.0, 0.0};
    for (int i = 0; i < N; ++i) as = as + (double)sg[i] * ccast<double>(a_vis[i]);
    R ed = R(0);
    for (int b = 0; b < Nb; ++b) ed += R(sg[bonds[b].x] * sg[bonds[b].y]);
    double xsum = 0.0;
    cpx<double> off = {0.0, 0.0};
    for (int g0 = 0; g0 < Nb; g0 += GB) {
        // the pass's bonds: spin of the first site (sign bits) and antiparallel bits
        // the pass reads table columns base .. base + GB - 1 at constant offsets:
        // the last pass is moved back to end at Nb, and its columns that the
        // previous pass took (below g0) are left out of the sum
        const bool fits = Nb >= GB;
        const int base = fits ? (g0 + GB <= Nb ? g0 : Nb - GB) : 0;
        uint32_t anti = 0u;
        cpx<R> pr[GB];
        R sv[GB];
        int ex = 0;  // one power-of-two scale for the pass's products
#pragma unroll
        for (int q = 0; q < GB; ++q) {
            const int b = base + q < Nb ? base + q : Nb - 1;
            const int sx = sg[bonds[b].x], sy = sg[bonds[b].y];
            sv[q] = R(sx);
            if (base + q >= g0 && base + q < Nb && sx != sy) anti |= 1u << q;
            pr[q] = ea[2 * b + (sx > 0 ? 0 : 1)];
        }
        for (int mc = 0; mc < M; mc += SYM_MC) {
            __syncwarp();
            for (int e = lane; e < 32 * SYM_MC; e += 32) {
                const int mm = e >> 5, cf = e & 31, wc = wb + 32 * wid + cf;  // th[mm][cf]
                th[e] = (wc < nc && mc + mm < M) ? theta[(size_t)wc * M + mc + mm]
                                                 : cpx<R>{R(0), R(0)};
            }
            __syncwarp();
            const int mlim = M - mc < SYM_MC ? M - mc : SYM_MC;
            for (int mm = 0; mm < mlim; ++mm) {
                const int m = mc + mm;
                const cpx<R> tv = th[mm * 32 + lane];
                const R ax = tv.x < R(0) ? -tv.x : tv.x;
                const R e = m_exp(R(-2) * ax), sgn = tv.x < R(0) ? R(-1) : R(1);
                R sn, cs;
                m_sincos(tv.y, &sn, &cs);
                const R hp = R(0.5) * (R(1) + e), hm = sgn * R(0.5) * (R(1) - e);
                const cpx<R> Cm = {hp * cs, hm * sn}, Sm = {hm * cs, hp * sn};
                if (g0 == 0) xsum += (double)ax;
                const cpx<R>* chr = ChT + (size_t)m * Nb + base;
                const cpx<R>* shr = ShT + (size_t)m * Nb + base;
                if (fits) {
#pragma unroll
                    for (int q = 0; q < GB; ++q) {
                        const cpx<R> ch = ldg(chr + q), sh = ldg(shr + q);  // same address in every lane
                        const cpx<R> x = Cm * ch, y = Sm * sh;
                        pr[q] = pr[q] * cpx<R>{x.x - sv[q] * y.x, x.y - sv[q] * y.y};
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < GB; ++q) {
                        const int qq = q < Nb ? q : Nb - 1;
                        const cpx<R> ch = ldg(chr + qq), sh = ldg(shr + qq);
                        const cpx<R> x = Cm * ch, y = Sm * sh;
                        pr[q] = pr[q] * cpx<R>{x.x - sv[q] * y.x, x.y - sv[q] * y.y};
                    }
                }
                if ((m & 15) == 15) {
                    // rescale by the largest: a product 2^-126 below it is
                    // negligible in the sum
                    R mx = R(0);
#pragma unroll
                    for (int q = 0; q < GB; ++q) mx = fmax(mx, fmax(fabs(pr[q].x), fabs(pr[q].y)));
                    int ee;
                    frexp(mx, &ee);
                    const R sc = ldexp(R(1), -ee);
#pragma unroll
                    for (int q = 0; q < GB; ++q) pr[q] = sc * pr[q];
                    ex += ee;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < GB; ++q)
            if ((anti >> q) & 1u)
                off = off + cpx<double>{ldexp((double)pr[q].x, ex), ldexp((double)pr[q].y, ex)};
    }
    if (valid) {
        const int s = w % B;
        const double edd = 0.25 * J * (double)ed;
        const cpx<double> ref = ccast<double>(lp_ref[s]);
        const cpx<double> lam = {as.x + M * 0.69314718055994530942 + xsum - ref.x, as.y - ref.y};
        const cpx<double> v = cexp_(ccast<double>(lp[w]) - ref);
        const double ia = 1.0 / a;
        const cpx<double> r = (ia * edd - (E0 * ia + Wp)) * v + (0.5 * J * ia) * (cexp_(lam) * off);
        hb[w] = ccast<R>(r);
    }
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

// Workspace: transformed configurations [4N][B][N] int8, log t_n at them
// [4N B], the rotation averages A [N][B]; with H also theta [4N B][M], the
// values (H' t_n)(s') / psi(s) [4N B] and HA [N][B].  Every part 256-byte
// aligned.
struct sym_ws {
    size_t lp, A, theta, hb, HA, total;
};

sym_ws ws_layout(const cr_ctx* c, int B, bool with_h) {
    const size_t N = c->N, cs = 2 * (size_t)rsize(c), nc = 4 * N * B;
    auto up = [](size_t x) { return ((x + 255) / 256) * 256; };
    sym_ws o = {};
    o.lp = up(nc * N);
    o.A = o.lp + up(nc * cs);
    o.total = o.A + N * B * cs;
    if (with_h) {
        o.theta = up(o.total);
        o.hb = o.theta + up(nc * c->M * cs);
        o.HA = o.hb + up(nc * cs);
        o.total = o.HA + N * B * cs;
    }
    return o;
}

// shared memory of sym_hprime_kernel
template <typename R> size_t sym_hprime_smem(const cr_ctx* c) {
    return (size_t)(c->Nb + (c->Nb & 1)) * sizeof(int2) + (size_t)4 * 32 * SYM_MC * sizeof(cpx<R>) +
           (size_t)128 * ((c->N + 3) & ~3);
}

// Opt sym_hprime_kernel into the shared memory of this context where it
// exceeds the default (called once per context, outside any capture).
cr_status sym_prepare_impl(cr_ctx* c) {
    const size_t s4 = sym_hprime_smem<float>(c), s8 = sym_hprime_smem<double>(c);
    cudaError_t e = cudaSuccess;
    if (s4 > 48 * 1024)
        e = cudaFuncSetAttribute(sym_hprime_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s4);
    if (e == cudaSuccess && s8 > 48 * 1024)
        e = cudaFuncSetAttribute(sym_hprime_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)s8);
    return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "sym_prepare: %s", cudaGetErrorString(e));
}

template <typename R>
cr_status launch_sym_hprime(cr_ctx* c, const void* params, const int8_t* sp, int nc, int B,
                            const cpx<R>* th, const cpx<R>* lp, const void* lp_ref,
                            const double* hp, cpx<R>* hb) {
    cr_status s = build_tables(c, params, 1);
    if (s != CR_OK) return s;
    const cr_tables& t = c->tab[1];
    const size_t sm = sym_hprime_smem<R>(c);
    CR_LAUNCH(c, CR_KERNEL_TARGET,
              sym_hprime_kernel<R><<<(unsigned)((nc + 127) / 128), 128, sm, c->stream>>>(
                  sp, th, lp, (const cpx<R>*)lp_ref, (const cpx<R>*)params, (const cpx<R>*)t.ChT,
                  (const cpx<R>*)t.ShT, (const cpx<R>*)t.ea, c->d_bonds, nc, B, c->N, c->M, c->Mp,
                  c->Nb, c->J, hp[0], hp[1], hp[2], hb));
    return cr_check_launch(c, "sym_hprime_kernel");
}

template <typename R>
cr_status btilde_t(cr_ctx* c, const cr_state* states, int Nm, const int8_t* spins,
                   const void* lp_ref, int B, const double* hp, unsigned char* ws, void* Bt,
                   void* HBt) {
    const int L = c->Lx, N = c->N;
    const bool h = HBt != nullptr;
    const sym_ws o = ws_layout(c, B, h);
    int8_t* sp = (int8_t*)ws;
    cpx<R>* lp = (cpx<R>*)(ws + o.lp);
    cpx<R>* A = (cpx<R>*)(ws + o.A);
    cpx<R>* th = h ? (cpx<R>*)(ws + o.theta) : nullptr;
    cpx<R>* hb = h ? (cpx<R>*)(ws + o.hb) : nullptr;
    cpx<R>* HA = h ? (cpx<R>*)(ws + o.HA) : nullptr;
    const int nc = 4 * N * B;
    const size_t np = (size_t)nc * N;
    CR_LAUNCH(c, CR_K_OTHER, sym_permute_kernel<<<(unsigned)((np + 255) / 256), 256, 0, c->stream>>>(spins, B, L, sp));
    const size_t nb = (size_t)N * B;
    const unsigned gb = (unsigned)((nb + 255) / 256);
    for (int n = 0; n < Nm; ++n) {
        cr_status s = launch_logpsi(c, states[n].params, sp, nc, th, lp);
        if (s != CR_OK) return s;
        if (h) {
            s = launch_sym_hprime<R>(c, states[n].params, sp, nc, B, th, lp, lp_ref, hp, hb);
            if (s != CR_OK) return s;
        }
        CR_LAUNCH(c, CR_K_OTHER, sym_rot_kernel<R><<<gb, 256, 0, c->stream>>>(
                                     lp, (const cpx<R>*)lp_ref, hb, N, B, A, HA));
        CR_LAUNCH(c, CR_K_OTHER, sym_dft_kernel<R><<<gb, 256, L * sizeof(cpx<R>), c->stream>>>(
                                     A, L, B, n, Nm, (cpx<R>*)Bt));
        if (h)
            CR_LAUNCH(c, CR_K_OTHER, sym_dft_kernel<R><<<gb, 256, L * sizeof(cpx<R>), c->stream>>>(
                                         HA, L, B, n, Nm, (cpx<R>*)HBt));
    }
    return cr_check_launch(c, h ? "sym_hbtilde" : "sym_btilde");
}

cr_status btilde_checked(cr_ctx* ctx, const char* name, const cr_state* states, int Nm,
                         const int8_t* spins, const void* logpsi_ref, int B, const double* hp,
                         void* workspace, size_t workspace_bytes, void* Bt_out, void* HBt_out) {
    CR_CHECK_ARG(ctx->Ly == ctx->Lx, "%s: needs a square L x L lattice", name);
    CR_CHECK_ARG(Nm >= 1 && B >= 1, "%s: Nm and B must be >= 1", name);
    CR_CHECK_ARG((size_t)4 * ctx->N * B <= (size_t)0x7fffffff &&
                     (size_t)4 * ctx->N * B * ctx->N / 256 < (size_t)0x7fffffff,
                 "%s: 4 N B too large", name);
    CR_CHECK_ARG(states && spins && logpsi_ref && workspace && Bt_out, "%s: null array", name);
    const size_t need = ws_layout(ctx, B, HBt_out != nullptr).total;
    CR_CHECK_ARG(workspace_bytes >= need, "%s: workspace of %zu bytes, need %zu", name,
                 workspace_bytes, need);
    for (int n = 0; n < Nm; ++n)
        CR_CHECK_ARG(states[n].params && !states[n].probe,
                     "%s: state %d: plain RBM states only (no probe factor)", name, n);
    unsigned char* ws = (unsigned char*)workspace;
    return ctx->prec == CR_FP64
               ? btilde_t<double>(ctx, states, Nm, spins, logpsi_ref, B, hp, ws, Bt_out, HBt_out)
               : btilde_t<float>(ctx, states, Nm, spins, logpsi_ref, B, hp, ws, Bt_out, HBt_out);
}

}  // namespace

cr_status sym_prepare(cr_ctx* c) { return sym_prepare_impl(c); }

extern "C" size_t sym_workspace_bytes(const cr_ctx* ctx, int B) {
    if (!ctx || B < 1) return 0;
    return ws_layout(ctx, B, false).total;
}

extern "C" size_t sym_h_workspace_bytes(const cr_ctx* ctx, int B) {
    if (!ctx || B < 1) return 0;
    return ws_layout(ctx, B, true).total;
}

extern "C" cr_status sym_btilde(cr_ctx* ctx, const cr_state* states, int Nm, const int8_t* spins,
                                const void* logpsi_ref, int B, void* workspace,
                                size_t workspace_bytes, void* Bt_out) {
    if (!ctx) return CR_EINVAL;
    return btilde_checked(ctx, "sym_btilde", states, Nm, spins, logpsi_ref, B, nullptr, workspace,
                          workspace_bytes, Bt_out, nullptr);
}

extern "C" cr_status sym_hbtilde(cr_ctx* ctx, const cr_state* states, int Nm, const int8_t* spins,
                                 const void* logpsi_ref, int B, const double* hprime,
                                 void* workspace, size_t workspace_bytes, void* Bt_out,
                                 void* HBt_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(hprime && hprime[1] != 0.0, "sym_hbtilde: needs hprime = {E0, a, W'}, a != 0");
    CR_CHECK_ARG(HBt_out, "sym_hbtilde: null HBt_out");
    return btilde_checked(ctx, "sym_hbtilde", states, Nm, spins, logpsi_ref, B, hprime, workspace,
                          workspace_bytes, Bt_out, HBt_out);
}
