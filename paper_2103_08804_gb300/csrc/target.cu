// The local target R(s) of the projected Chebyshev recursion (Sec. III, last
// paragraph) and the moment / Krylov columns (Secs. II, IV).
//
// Both apply H' = (H - E0)/a - W' to a state v at a sample s, relative to a
// reference amplitude psi_ref(s):
//   (H v)(s) = sum_b [(J/4) s_i s_j v(s) + (J/2)[s_i != s_j] v(s^{ij})]   (Sec. V)
// One warp per sample.  Lanes take the antiparallel bonds of the sample
// (compacted with a ballot) and run over the hidden units sequentially,
// forming the exchanged amplitude relative to the reference amplitude with
// no division:
//   v(s^{ij}) / psi_ref(s) = exp(a.s - 2 s_i (a_i - a_i') + X + M ln 2 - log psi_ref(s))
//                            prod_m (C_m cosh D_m - s_i S_m sinh D_m),
// C_m, S_m = cosh, sinh theta_m times e^{-|Re theta_m|} and X = sum_m |Re theta_m|,
// from the transposed bond tables [Mp][Nb] (consecutive lanes read
// consecutive bonds).  The samples are drawn from |psi_n|^2, not from
// |v|^2, so a sample can sit at a node of v (cosh theta_m = 0); a ratio to
// v(s), as with tanh theta_m, would divide by it there, while every factor
// above stays bounded.
#include <math.h>

#include "common.cuh"

struct probe_desc {
    int on;
    double qx, qy;
};

template <typename R>
struct hp_args {
    const int8_t* spins;
    const cpx<R>* L_prev;    // [B] log RBM(prev) at s
    const cpx<R>* th_prev;   // [B][M] theta of prev at s
    const cpx<R>* a_prev;    // [N] visible biases of prev
    const cpx<R>* L_ref;     // [B] log psi_ref at s
    const cpx<R>* L_prev2;   // [B] log RBM(prev2) at s, or null
    const cpx<R>* ChT;
    const cpx<R>* ShT;
    const cpx<R>* ea;
    const int2* bonds;
    probe_desc pr, pr2, prm;  // probe of prev, of prev2, and of the moment bra
    int want_E;
    const double* beta_a;    // complex128: scales E (times ka) and out2
    const double* beta_b;    // complex128: -beta_b scales V2, or null
    double ka;
    R J, E0, a, Wp;
    int B, N, Lx, M, Mp, Nb;
    cpx<R>* out1;            // c1 E + c2 V2  (R or HB), or null
    cpx<R>* out2;            // cB V          (B column), or null
    cpx<R>* mu_terms;        // conj(f_moment) out2, or null
};

// f_q(s) = N^{-1/2} sum_r e^{-i q.r} s_r / 2, reduced over the warp.
template <typename R>
CR_D cpx<R> probe_value(const int8_t* sg, int N, int Lx, double qx, double qy, int lane) {
    cpx<R> acc = {R(0), R(0)};
    for (int r = lane; r < N; r += 32) {
        R sn, cs;
        m_sincos(R(qx * (r % Lx) + qy * (r / Lx)), &sn, &cs);
        acc = acc + R(sg[r]) * cpx<R>{cs, -sn};
    }
    return R(0.5) * m_rsqrt(R(N)) * warp_sum(acc);
}

template <typename R>
CR_D cpx<R> phase(int r, int Lx, double qx, double qy) {
    R sn, cs;
    m_sincos(R(qx * (r % Lx) + qy * (r / Lx)), &sn, &cs);
    return {cs, -sn};
}

template <typename R>
__global__ void __launch_bounds__(128) hprime_kernel(hp_args<R> A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int2* bonds = (int2*)smem_raw;                                   // [Nb]
    cpx<R>* Tall = (cpx<R>*)(bonds + A.Nb + (A.Nb & 1));             // [4][2 Mp]: C, S
    int8_t* sgall = (int8_t*)(Tall + 8 * A.Mp);                      // [4][N]
    int16_t* lstall = (int16_t*)(sgall + 4 * ((A.N + 1) & ~1));      // [4][Nb]
    for (int e = threadIdx.x; e < A.Nb; e += blockDim.x) bonds[e] = A.bonds[e];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int w = blockIdx.x * 4 + wid;
    cpx<R>* Cm = Tall + wid * 2 * A.Mp;
    cpx<R>* Sm = Cm + A.Mp;
    int8_t* sg = sgall + wid * ((A.N + 1) & ~1);
    int16_t* lst = lstall + wid * A.Nb;
    double xsum = 0.0;             // sum_m |Re theta_m| (lane partial)
    cpx<double> asg = {0.0, 0.0};  // a . s (lane partial)
    if (w < A.B) {
        for (int i = lane; i < A.N; i += 32) {
            const int8_t si = A.spins[(size_t)w * A.N + i];
            sg[i] = si;
            if (A.want_E) asg = asg + (double)si * ccast<double>(A.a_prev[i]);
        }
        if (A.want_E)
            for (int m = lane; m < A.M; m += 32) {
                // cosh and sinh of theta times e^{-|Re theta|}: with e = e^{-2|x|},
                // C = ((1 + e) cos y, sg (1 - e) sin y) / 2, S = (sg (1 - e) cos y, (1 + e) sin y) / 2
                const cpx<R> th = A.th_prev[(size_t)w * A.M + m];
                const R ax = th.x < R(0) ? -th.x : th.x, sgn = th.x < R(0) ? R(-1) : R(1);
                const R e = m_exp(R(-2) * ax);
                R sn, cs;
                m_sincos(th.y, &sn, &cs);
                const R p = R(0.5) * (R(1) + e), q = R(0.5) * sgn * (R(1) - e);
                Cm[m] = {p * cs, q * sn};
                Sm[m] = {q * cs, p * sn};
                xsum += (double)ax;
            }
    }
    __syncthreads();
    if (w >= A.B) return;

    const cpx<R> one = {R(1), R(0)};
    const cpx<R> fs = A.pr.on ? probe_value<R>(sg, A.N, A.Lx, A.pr.qx, A.pr.qy, lane) : one;
    // Amplitude ratios of two different RBMs, exp(log t(s) - log psi(s)), and
    // the products with the beta coefficients are formed in float64: the RBM
    // amplitudes carry no normalisation, so a ratio can leave the float32
    // range while the product beta * ratio stays moderate.
    const cpx<double> V = cexp_(ccast<double>(A.L_prev[w] - A.L_ref[w]));
    cpx<double> E = {0.0, 0.0};
    if (A.want_E) {
        // diagonal part and the list of antiparallel bonds
        R ed = R(0);
        int n_anti = 0;
        for (int b0 = 0; b0 < A.Nb; b0 += 32) {
            int b = b0 + lane;
            bool anti = false;
            if (b < A.Nb) {
                int2 bd = bonds[b];
                int p = sg[bd.x] * sg[bd.y];
                ed += R(p);
                anti = p < 0;
            }
            unsigned msk = __ballot_sync(0xffffffffu, anti);
            if (anti) lst[n_anti + __popc(msk & ((1u << lane) - 1u))] = (int16_t)b;
            n_anti += __popc(msk);
        }
        __syncwarp();
        ed = R(0.25) * A.J * warp_sum(ed);
        cpx<double> off = {0.0, 0.0};
        const R inv_sqrt_n = m_rsqrt(R(A.N));
        xsum = warp_sum(xsum);
        asg = warp_sum(asg);
        // two bonds per lane at a time (k and k + 32 of the list): two
        // independent product chains share the C_m, S_m reads and keep twice
        // the table loads in flight; the sum runs in the list's order
        for (int k0 = 0; k0 < n_anti; k0 += 64) {
            int kk[2], bb[2], ex[2] = {0, 0};
            R sv[2];
            cpx<R> pr[2];
            const cpx<R>* chc[2];
            const cpx<R>* shc[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                kk[u] = k0 + 32 * u + lane;
                bb[u] = kk[u] < n_anti ? lst[kk[u]] : 0;  // bond 0 as a placeholder
                const int si = sg[bonds[bb[u]].x];
                sv[u] = R(si);
                pr[u] = A.ea[2 * bb[u] + (si > 0 ? 0 : 1)];
                chc[u] = A.ChT + bb[u];
                shc[u] = A.ShT + bb[u];
            }
            // the products of M factors are kept as pr * 2^ex, renormalised
            // every 16 factors, so they cannot overflow or underflow float32
            for (int m = 0; m < A.M; ++m) {
                const cpx<R> cm = Cm[m], sm = Sm[m];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const cpx<R> ch = ldg(chc[u] + (size_t)m * A.Nb), sh = ldg(shc[u] + (size_t)m * A.Nb);
                    const cpx<R> c1 = cm * ch, s1 = sm * sh;
                    // cosh(theta - s D) e^{-|Re theta|}
                    pr[u] = pr[u] * cpx<R>{c1.x - sv[u] * s1.x, c1.y - sv[u] * s1.y};
                }
                if ((m & 15) == 15) {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        int e;
                        frexp(fmax(fabs(pr[u].x), fabs(pr[u].y)), &e);
                        pr[u] = {ldexp(pr[u].x, -e), ldexp(pr[u].y, -e)};
                        ex[u] += e;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                if (kk[u] >= n_anti) continue;
                if (A.pr.on) {
                    // f(s^{ij}) = f(s) + s (e^{-iq.r_i'} - e^{-iq.r_i}) / sqrt(N)
                    const int2 bd = bonds[bb[u]];
                    cpx<R> d = phase<R>(bd.y, A.Lx, A.pr.qx, A.pr.qy) -
                               phase<R>(bd.x, A.Lx, A.pr.qx, A.pr.qy);
                    pr[u] = (fs + (sv[u] * inv_sqrt_n) * d) * pr[u];
                }
                off = off + cpx<double>{ldexp((double)pr[u].x, ex[u]), ldexp((double)pr[u].y, ex[u])};
            }
        }
        off = warp_sum(off);
        const double ia = 1.0 / A.a;
        const cpx<double> fsd = ccast<double>(fs);
        // the exchanged amplitudes relative to psi_ref(s)
        const cpx<double> base = asg - ccast<double>(A.L_ref[w]) +
                                 cpx<double>{xsum + A.M * 0.6931471805599453, 0.0};
        const cpx<double> offr = cexp_(base) * off;
        E = ia * ((double)ed * (fsd * V) + (0.5 * A.J) * offr) - (A.E0 * ia + A.Wp) * (fsd * V);
    }
    const cpx<double> ba = {A.beta_a[0], A.beta_a[1]};
    const cpx<double> c1 = A.ka * ba;
    const cpx<double> c2 = A.beta_b ? cpx<double>{-A.beta_b[0], -A.beta_b[1]}
                                    : cpx<double>{0.0, 0.0};
    cpx<double> o1 = c1 * E;
    if (A.L_prev2 && lane == 0 && !A.pr2.on)
        o1 = o1 + c2 * cexp_(ccast<double>(A.L_prev2[w] - A.L_ref[w]));
    // the prev2 probe factor and the moment bra need their own warp reductions
    if (A.L_prev2 && A.pr2.on) {
        cpx<R> f2 = probe_value<R>(sg, A.N, A.Lx, A.pr2.qx, A.pr2.qy, lane);
        if (lane == 0)
            o1 = o1 + c2 * (ccast<double>(f2) * cexp_(ccast<double>(A.L_prev2[w] - A.L_ref[w])));
    }
    const cpx<double> o2 = ba * (ccast<double>(fs) * V);
    if (lane == 0) {
        if (A.out1) A.out1[w] = ccast<R>(o1);
        if (A.out2) A.out2[w] = ccast<R>(o2);
    }
    if (A.mu_terms) {
        cpx<R> fm = probe_value<R>(sg, A.N, A.Lx, A.prm.qx, A.prm.qy, lane);
        if (lane == 0) A.mu_terms[w] = ccast<R>(cmulc(ccast<double>(fm), o2));
    }
}

// mu = sum_s terms[s] / B, summed in float64 by one CTA in a fixed order.
template <typename R>
__global__ void mean_kernel(const cpx<R>* __restrict__ terms, int B, double* __restrict__ out) {
    __shared__ double sx[32], sy[32];
    double x = 0, y = 0;
    for (int s = threadIdx.x; s < B; s += blockDim.x) {
        x += (double)terms[s].x;
        y += (double)terms[s].y;
    }
    x = warp_sum(x);
    y = warp_sum(y);
    if ((threadIdx.x & 31) == 0) {
        sx[threadIdx.x >> 5] = x;
        sy[threadIdx.x >> 5] = y;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tx = 0, ty = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            tx += sx[k];
            ty += sy[k];
        }
        out[0] = tx / B;
        out[1] = ty / B;
    }
}

// Shared memory of hprime_kernel for a context, and the opt-in above the
// 48 KB default (set once per context, outside any hot call).
template <typename R>
static size_t hprime_smem(const cr_ctx* c) {
    return (c->Nb + (c->Nb & 1)) * sizeof(int2) + 8 * c->Mp * sizeof(cpx<R>) +
           4 * ((c->N + 1) & ~1) + 4 * c->Nb * sizeof(int16_t);
}

cr_status target_prepare(cr_ctx* c) {
    const size_t sm = c->prec == CR_FP64 ? hprime_smem<double>(c) : hprime_smem<float>(c);
    if (sm <= 48 * 1024) return CR_OK;
    cudaError_t e = c->prec == CR_FP64
                        ? cudaFuncSetAttribute(hprime_kernel<double>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)
                        : cudaFuncSetAttribute(hprime_kernel<float>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "target_prepare: %s", cudaGetErrorString(e));
}

template <typename R>
static cr_status launch_hprime(cr_ctx* c, hp_args<R>& A) {
    const cr_tables& t = c->tab[1];
    A.ChT = (const cpx<R>*)t.ChT;
    A.ShT = (const cpx<R>*)t.ShT;
    A.ea = (const cpx<R>*)t.ea;
    A.bonds = c->d_bonds;
    A.N = c->N;
    A.Lx = c->Lx;
    A.M = c->M;
    A.Mp = c->Mp;
    A.Nb = c->Nb;
    A.J = (R)c->J;
    const size_t sm = hprime_smem<R>(c);
    CR_LAUNCH(c, CR_KERNEL_TARGET, hprime_kernel<R><<<(A.B + 3) / 4, 128, sm, c->stream>>>(A));
    return cr_check_launch(c, "hprime_kernel");
}

static probe_desc pd(const cr_state* s) { return probe_desc{s->probe != 0, s->qx, s->qy}; }

template <typename R>
static cr_status target_t(cr_ctx* c, const cr_target* tg, const int8_t* spins, const void* lpn,
                          int B, void* R_out, double* mean_out) {
    cr_status s = build_tables(c, tg->prev.params, 1);
    if (s != CR_OK) return s;
    cpx<R>* lp = (cpx<R>*)c->lp_tmp;
    s = launch_logpsi(c, tg->prev.params, spins, B, c->theta_tmp, lp);
    if (s != CR_OK) return s;
    if (tg->n >= 2) {
        s = launch_logpsi(c, tg->prev2.params, spins, B, nullptr, lp + c->max_walkers);
        if (s != CR_OK) return s;
    }
    hp_args<R> A = {};
    A.spins = spins;
    A.L_prev = lp;
    A.th_prev = (const cpx<R>*)c->theta_tmp;
    A.a_prev = (const cpx<R>*)tg->prev.params;
    A.L_ref = (const cpx<R>*)lpn;
    A.L_prev2 = tg->n >= 2 ? lp + c->max_walkers : nullptr;
    A.pr = pd(&tg->prev);
    A.pr2 = pd(&tg->prev2);
    A.want_E = 1;
    A.ka = tg->n == 1 ? 1.0 : 2.0;
    A.beta_a = tg->beta_prev;
    A.beta_b = tg->n >= 2 ? tg->beta_prev2 : nullptr;
    A.E0 = (R)tg->E0;
    A.a = (R)tg->a;
    A.Wp = (R)tg->Wp;
    A.B = B;
    A.out1 = (cpx<R>*)R_out;
    s = launch_hprime<R>(c, A);
    if (s != CR_OK || !mean_out) return s;
    CR_LAUNCH(c, CR_K_OTHER, mean_kernel<R><<<1, 1024, 0, c->stream>>>((const cpx<R>*)R_out, B, mean_out));
    return cr_check_launch(c, "mean_kernel");
}

extern "C" cr_status cheb_local_target(cr_ctx* ctx, const cr_target* tg, const int8_t* spins,
                                       const void* logpsi_n, int B, void* R_out,
                                       double* mean_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(tg && tg->prev.params, "cheb_local_target: null target");
    CR_CHECK_ARG(tg->n >= 1, "cheb_local_target: n must be >= 1");
    CR_CHECK_ARG(tg->n == 1 || tg->prev2.params, "cheb_local_target: null prev2 for n >= 2");
    CR_CHECK_ARG(tg->beta_prev && (tg->n == 1 || tg->beta_prev2), "cheb_local_target: null beta");
    CR_CHECK_ARG(tg->a != 0.0, "cheb_local_target: a == 0");
    CR_CHECK_ARG(B >= 0 && B <= ctx->max_walkers, "cheb_local_target: B=%d outside [0, %d]", B,
                 ctx->max_walkers);
    if (B == 0) return CR_OK;
    CR_CHECK_ARG(spins && logpsi_n && R_out, "cheb_local_target: null array");
    return ctx->prec == CR_FP64 ? target_t<double>(ctx, tg, spins, logpsi_n, B, R_out, mean_out)
                                : target_t<float>(ctx, tg, spins, logpsi_n, B, R_out, mean_out);
}

template <typename R>
static cr_status moment_t(cr_ctx* c, const cr_state* st, const double* beta, double qx, double qy,
                          const int8_t* spins, const void* lpref, int B, const double* hp,
                          void* Bcol, void* HBcol, double* mu_out) {
    cr_status s;
    if (HBcol) {
        s = build_tables(c, st->params, 1);
        if (s != CR_OK) return s;
    }
    cpx<R>* lp = (cpx<R>*)c->lp_tmp;
    s = launch_logpsi(c, st->params, spins, B, HBcol ? c->theta_tmp : nullptr, lp);
    if (s != CR_OK) return s;
    hp_args<R> A = {};
    A.spins = spins;
    A.L_prev = lp;
    A.th_prev = (const cpx<R>*)c->theta_tmp;
    A.a_prev = (const cpx<R>*)st->params;
    A.L_ref = (const cpx<R>*)lpref;
    A.pr = pd(st);
    A.prm = probe_desc{1, qx, qy};
    A.want_E = HBcol != nullptr;
    A.ka = 1.0;
    A.beta_a = beta;
    A.beta_b = nullptr;
    if (hp) {
        A.E0 = (R)hp[0];
        A.a = (R)hp[1];
        A.Wp = (R)hp[2];
    } else {
        A.a = R(1);
    }
    A.B = B;
    A.out1 = (cpx<R>*)HBcol;
    A.out2 = (cpx<R>*)Bcol;
    A.mu_terms = mu_out ? lp + c->max_walkers : nullptr;
    s = launch_hprime<R>(c, A);
    if (s != CR_OK || !mu_out) return s;
    CR_LAUNCH(c, CR_K_OTHER, mean_kernel<R><<<1, 1024, 0, c->stream>>>(lp + c->max_walkers, B, mu_out));
    return cr_check_launch(c, "mean_kernel");
}

extern "C" cr_status cheb_moment(cr_ctx* ctx, const cr_state* st, const double* beta, double qx,
                                 double qy, const int8_t* spins, const void* logpsi_ref, int B,
                                 const double* hprime, void* Bcol, void* HBcol, double* mu_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(st && st->params && beta, "cheb_moment: null state or beta");
    CR_CHECK_ARG(!HBcol || (hprime && hprime[1] != 0.0), "cheb_moment: HBcol needs hprime, a != 0");
    CR_CHECK_ARG(B >= 0 && B <= ctx->max_walkers, "cheb_moment: B=%d outside [0, %d]", B,
                 ctx->max_walkers);
    if (B == 0) return CR_OK;
    CR_CHECK_ARG(spins && logpsi_ref, "cheb_moment: null spins or logpsi_ref");
    return ctx->prec == CR_FP64
               ? moment_t<double>(ctx, st, beta, qx, qy, spins, logpsi_ref, B, hprime, Bcol, HBcol,
                                  mu_out)
               : moment_t<float>(ctx, st, beta, qx, qy, spins, logpsi_ref, B, hprime, Bcol, HBcol,
                                 mu_out);
}
