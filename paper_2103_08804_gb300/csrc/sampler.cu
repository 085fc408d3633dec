// Metropolis sampling of |psi_s|^2 (Sec. III) with S^z-conserving exchange
// moves on nearest-neighbour bonds.
//
// One warp per walker.  Lane l owns the KPL hidden units j = 32 k + l
// (k < KPL) of the padded width Mp = 32 KPL and keeps theta and tanh(theta)
// for them in registers, so that every table read of a proposal is 32
// consecutive entries (two 128-byte lines per load instruction).  The amplitude ratio of a proposal is the
// product over hidden units of (cosh D - s tanh(theta) sinh D) from the bond
// tables, so the inner loop is complex FMA only; accepted moves update theta
// and tanh(theta) by the same addition formulas.  Proposals on parallel
// bonds are no-ops (rejected) and cost a shared-memory read.
#include "common.cuh"

template <typename R, int KPL>
__global__ void __launch_bounds__(128) sweep_kernel(
    const cpx<R>* __restrict__ prm, int8_t* __restrict__ spins, cpx<R>* __restrict__ theta, int B,
    int N, int M, int Mp, int Nb, const int2* __restrict__ bonds_g, const cpx<R>* __restrict__ Dt,
    const cpx<R>* __restrict__ Cht, const cpx<R>* __restrict__ Sht, const cpx<R>* __restrict__ ea,
    int n_prop, uint32_t k0, uint32_t k1, unsigned long long counter,
    const unsigned long long* __restrict__ dcounter, cpx<R>* __restrict__ logpsi_out,
    cpx<R>* __restrict__ tanh_out, int32_t* __restrict__ n_acc) {
    if (dcounter) counter = *dcounter;  // stream position kept on the device
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int2* bonds = (int2*)smem_raw;                       // [Nb]
    int8_t* sg_all = (int8_t*)(bonds + Nb);              // [4][N]
    for (int e = threadIdx.x; e < Nb; e += blockDim.x) bonds[e] = bonds_g[e];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int w = blockIdx.x * 4 + wid;
    int8_t* sg = sg_all + wid * N;
    if (w < B)
        for (int i = lane; i < N; i += 32) sg[i] = spins[(size_t)w * N + i];
    __syncthreads();
    if (w >= B) return;

    cpx<R> th[KPL], T[KPL];
#pragma unroll
    for (int k = 0; k < KPL; ++k) {
        int j = 32 * k + lane;
        th[k] = j < M ? theta[(size_t)w * M + j] : cpx<R>{R(0), R(0)};
        T[k] = ctanh_(th[k]);
    }
    int nacc = 0;
    uint4 rnd = make_uint4(0, 0, 0, 0);
    for (int p = 0; p < n_prop; ++p) {
        if ((p & 63) == 0) {
            unsigned long long step = counter + (unsigned long long)(p >> 1) + lane;
            rnd = philox4x32_10(make_uint4((uint32_t)w, (uint32_t)step, (uint32_t)(step >> 32), 0u),
                                k0, k1);
        }
        const int src = (p >> 1) & 31;
        const uint32_t ub = __shfl_sync(0xffffffffu, (p & 1) ? rnd.z : rnd.x, src);
        const uint32_t ua = __shfl_sync(0xffffffffu, (p & 1) ? rnd.w : rnd.y, src);
        const int b = (int)__umulhi(ub, (uint32_t)Nb);
        const int2 bd = bonds[b];
        const int si = sg[bd.x];
        if (si == sg[bd.y]) continue;  // parallel: no-op, counts as rejected
        const R s = R(si);
        const cpx<R>* chr = Cht + (size_t)b * Mp + lane;
        const cpx<R>* shr = Sht + (size_t)b * Mp + lane;
        cpx<R> ch[KPL], sh[KPL], f[KPL];
        cpx<R> pl = {R(1), R(0)};
#pragma unroll
        for (int k = 0; k < KPL; ++k) {
            ch[k] = ldg(chr + 32 * k);
            sh[k] = ldg(shr + 32 * k);
            cpx<R> ts = T[k] * sh[k];
            f[k] = {ch[k].x - s * ts.x, ch[k].y - s * ts.y};
            pl = pl * f[k];
        }
        cpx<R> pw = warp_prod(pl);
        pw.x = __shfl_sync(0xffffffffu, pw.x, 0);  // one value for the whole warp
        pw.y = __shfl_sync(0xffffffffu, pw.y, 0);
        const cpx<R> e = ea[2 * b + (si > 0 ? 0 : 1)];
        const R ratio2 = abs2(e) * abs2(pw);
        const R u = (R(ua >> 9) + R(0.5)) * R(1.1920928955078125e-07);
        if (u < ratio2) {
            const cpx<R>* dr = Dt + (size_t)b * Mp + lane;
#pragma unroll
            for (int k = 0; k < KPL; ++k) {
                cpx<R> d = ldg(dr + 32 * k);
                th[k] = {th[k].x - s * d.x, th[k].y - s * d.y};
                cpx<R> tc = T[k] * ch[k];
                T[k] = cdiv(cpx<R>{tc.x - s * sh[k].x, tc.y - s * sh[k].y}, f[k]);
            }
            __syncwarp();
            if (lane == 0) {
                sg[bd.x] = (int8_t)(-si);
                sg[bd.y] = (int8_t)si;
            }
            __syncwarp();
            ++nacc;
        }
    }
    __syncwarp();
    for (int i = lane; i < N; i += 32) spins[(size_t)w * N + i] = sg[i];
    cpx<R> lp = {R(0), R(0)};
#pragma unroll
    for (int k = 0; k < KPL; ++k) {
        int j = 32 * k + lane;
        if (j < M) {
            theta[(size_t)w * M + j] = th[k];
            lp = lp + clncosh2_(th[k]);
            if (tanh_out) tanh_out[(size_t)w * M + j] = ctanh_(th[k]);
        }
    }
    for (int i = lane; i < N; i += 32) lp = lp + R(sg[i]) * prm[i];
    lp = warp_sum(lp);
    if (lane == 0) {
        if (logpsi_out) logpsi_out[w] = lp;
        if (n_acc) n_acc[w] = nacc;
    }
}

// Advance a device-resident stream position (after the sweep that used it).
__global__ void advance_counter_kernel(unsigned long long* ctr, unsigned long long calls) {
    *ctr += calls;
}

template <typename R>
static cr_status sweep_t(cr_ctx* c, const void* params, int8_t* spins, void* theta, int B,
                         int n_prop, uint64_t seed, uint64_t counter, const uint64_t* dcounter,
                         void* logpsi_out, void* tanh_out, int32_t* n_acc) {
    const cr_tables& t = c->tab[0];
    const int kpl = c->Mp / 32;
    size_t sm = c->Nb * sizeof(int2) + 4 * c->N;
    dim3 grid((B + 3) / 4);
#define LAUNCH(K)                                                                                  \
    CR_LAUNCH(c, CR_KERNEL_SWEEP, sweep_kernel<R, K><<<grid, 128, sm, c->stream>>>(                                             \
        (const cpx<R>*)params, spins, (cpx<R>*)theta, B, c->N, c->M, c->Mp, c->Nb, c->d_bonds,     \
        (const cpx<R>*)t.D, (const cpx<R>*)t.Ch, (const cpx<R>*)t.Sh, (const cpx<R>*)t.ea, n_prop, \
        (uint32_t)seed, (uint32_t)(seed >> 32), (unsigned long long)counter,                        \
        (const unsigned long long*)dcounter, (cpx<R>*)logpsi_out, (cpx<R>*)tanh_out, n_acc))
    switch (kpl) {
        case 1: LAUNCH(1); break;
        case 2: LAUNCH(2); break;
        case 4: LAUNCH(4); break;
        case 8: LAUNCH(8); break;
        default: LAUNCH(16); break;
    }
#undef LAUNCH
    return cr_check_launch(c, "sweep_kernel");
}

extern "C" cr_status mc_sweep(cr_ctx* ctx, const cr_state* st, int8_t* spins, void* theta, int B,
                              int n_sweeps, cr_philox* rng, void* logpsi_out, void* tanh_out,
                              int32_t* n_accepted) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(st && st->params, "mc_sweep: null state");
    CR_CHECK_ARG(!st->probe, "mc_sweep: the sampled state must be a plain RBM");
    CR_CHECK_ARG(B >= 0 && B <= ctx->max_walkers, "mc_sweep: B=%d outside [0, %d]", B,
                 ctx->max_walkers);
    CR_CHECK_ARG(n_sweeps >= 0, "mc_sweep: n_sweeps < 0");
    CR_CHECK_ARG(rng, "mc_sweep: null rng");
    CR_CHECK_ARG(ctx->Mp <= 512, "mc_sweep: M > 512 not supported");
    const int n_prop = n_sweeps * ctx->N;
    const uint64_t calls = (uint64_t)(n_prop + 1) / 2;
    if (B > 0) {
        CR_CHECK_ARG(spins && theta, "mc_sweep: null spins or theta");
        cr_status s = build_tables(ctx, st->params, 0);
        if (s != CR_OK) return s;
        s = ctx->prec == CR_FP64
                ? sweep_t<double>(ctx, st->params, spins, theta, B, n_prop, rng->seed,
                                  rng->counter, rng->device_counter, logpsi_out, tanh_out,
                                  n_accepted)
                : sweep_t<float>(ctx, st->params, spins, theta, B, n_prop, rng->seed,
                                 rng->counter, rng->device_counter, logpsi_out, tanh_out,
                                 n_accepted);
        if (s != CR_OK) return s;
    }
    if (rng->device_counter) {
        CR_LAUNCH(ctx, CR_K_OTHER, advance_counter_kernel<<<1, 1, 0, ctx->stream>>>(
                                       (unsigned long long*)rng->device_counter, calls));
        return cr_check_launch(ctx, "advance_counter_kernel");
    }
    rng->counter += calls;
    return CR_OK;
}
