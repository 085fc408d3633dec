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
// configurations, one warp each (Sec. V bonds).  With x_m = Re theta_m(s'),
// C_m = cosh(theta_m) e^{-|x_m|} and S_m = sinh(theta_m) e^{-|x_m|} (both of
// modulus <= 1),
//   t_n(s'^{ij}) / psi(s) = e^{Lam} ea_b prod_m (C_m cosh D_bm - s_i S_m sinh D_bm),
//   Lam = a.s' + M log 2 + sum_m |x_m| - log psi(s),
// from cosh(theta - s D) = cosh theta cosh D - s sinh theta sinh D and the
// bond tables D_bm, ea_b of t_n; the product is renormalised every 16 factors
// and Lam, the diagonal part and the sums are formed in float64.
template <typename R>
__global__ void __launch_bounds__(128) sym_hprime_kernel(
    const int8_t* __restrict__ sp, const cpx<R>* __restrict__ theta, const cpx<R>* __restrict__ lp,
    const cpx<R>* __restrict__ lp_ref, const cpx<R>* __restrict__ a_vis,
    const cpx<R>* __restrict__ ChT, const cpx<R>* __restrict__ ShT, const cpx<R>* __restrict__ ea,
    const int2* __restrict__ bonds_g, int nc, int B, int N, int M, int Mp, int Nb, double J,
    double E0, double a, double Wp, cpx<R>* __restrict__ hb) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int2* bonds = (int2*)smem_raw;                                   // [Nb]
    cpx<R>* CSall = (cpx<R>*)(bonds + Nb + (Nb & 1));                // [4][2][Mp]
    int8_t* sgall = (int8_t*)(CSall + 8 * Mp);                       // [4][N]
    int16_t* lstall = (int16_t*)(sgall + 4 * ((N + 1) & ~1));       // [4][Nb]
    for (int e = threadIdx.x; e < Nb; e += blockDim.x) bonds[e] = bonds_g[e];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int w = blockIdx.x * 4 + wid;
    cpx<R>* C = CSall + 2 * wid * Mp;
    cpx<R>* S = C + Mp;
    int8_t* sg = sgall + wid * ((N + 1) & ~1);
    int16_t* lst = lstall + wid * Nb;
    double xsum = 0.0;
    cpx<double> as = {0.0, 0.0};
    if (w < nc) {
        for (int i = lane; i < N; i += 32) {
            sg[i] = sp[(size_t)w * N + i];
            as = as + (double)sg[i] * ccast<double>(a_vis[i]);
        }
        for (int m = lane; m < M; m += 32) {
            const cpx<R> th = theta[(size_t)w * M + m];
            const R ax = th.x < R(0) ? -th.x : th.x;
            const R e = m_exp(R(-2) * ax), sgn = th.x < R(0) ? R(-1) : R(1);
            R sn, cs;
            m_sincos(th.y, &sn, &cs);
            const R hp = R(0.5) * (R(1) + e), hm = sgn * R(0.5) * (R(1) - e);
            C[m] = {hp * cs, hm * sn};
            S[m] = {hm * cs, hp * sn};
            xsum += (double)ax;
        }
    }
    __syncthreads();
    if (w >= nc) return;
    xsum = warp_sum(xsum);
    as = warp_sum(as);

    R ed = R(0);
    int n_anti = 0;
    for (int b0 = 0; b0 < Nb; b0 += 32) {
        const int b = b0 + lane;
        bool anti = false;
        if (b < Nb) {
            const int2 bd = bonds[b];
            const int p = sg[bd.x] * sg[bd.y];
            ed += R(p);
            anti = p < 0;
        }
        const unsigned msk = __ballot_sync(0xffffffffu, anti);
        if (anti) lst[n_anti + __popc(msk & ((1u << lane) - 1u))] = (int16_t)b;
        n_anti += __popc(msk);
    }
    __syncwarp();
    const double edd = 0.25 * J * (double)warp_sum(ed);
    cpx<double> off = {0.0, 0.0};
    for (int k = lane; k < n_anti; k += 32) {
        const int b = lst[k];
        const int si = sg[bonds[b].x];
        const R s = R(si);
        cpx<R> pr = ea[2 * b + (si > 0 ? 0 : 1)];
        int ex = 0;
        for (int m = 0; m < M; ++m) {
            const cpx<R> ch = ChT[(size_t)m * Nb + b], sh = ShT[(size_t)m * Nb + b];
            const cpx<R> u = C[m] * ch, v = S[m] * sh;
            pr = pr * cpx<R>{u.x - s * v.x, u.y - s * v.y};
            if ((m & 15) == 15) {
                int e;
                frexp(fmax(fabs(pr.x), fabs(pr.y)), &e);
                pr = {ldexp(pr.x, -e), ldexp(pr.y, -e)};
                ex += e;
            }
        }
        off = off + cpx<double>{ldexp((double)pr.x, ex), ldexp((double)pr.y, ex)};
    }
    off = warp_sum(off);
    if (lane == 0) {
        const int s = w % B;
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

template <typename R>
cr_status launch_sym_hprime(cr_ctx* c, const void* params, const int8_t* sp, int nc, int B,
                            const cpx<R>* th, const cpx<R>* lp, const void* lp_ref,
                            const double* hp, cpx<R>* hb) {
    cr_status s = build_tables(c, params, 1);
    if (s != CR_OK) return s;
    const cr_tables& t = c->tab[1];
    const size_t sm = (c->Nb + (c->Nb & 1)) * sizeof(int2) + 8 * (size_t)c->Mp * sizeof(cpx<R>) +
                      4 * ((c->N + 1) & ~1) + 4 * c->Nb * sizeof(int16_t);
    CR_LAUNCH(c, CR_KERNEL_TARGET,
              sym_hprime_kernel<R><<<(unsigned)((nc + 3) / 4), 128, sm, c->stream>>>(
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
