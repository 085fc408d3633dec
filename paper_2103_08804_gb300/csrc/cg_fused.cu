// The whole matrix-free CG solve of the natural-gradient update (Sec. III),
//   (S + lambda I) x = F,   S v = (1/B) sum_s conj(O_s) ((O_s - Obar) . v),
// in ONE persistent kernel for CR_MIXED contexts: one CTA per SM, a bounded
// grid barrier between phases, the two O-contractions on the tensor cores
// (tcgen05, bf16 splits, float32 accumulation in TMEM) and the CG vectors in
// float64.
//
// With O_s = [sigma_s | T_s | sigma_s (x) T_s] (T = tanh theta) and
// v = [va | vb | V]:
//   u_s  = (O_s . v) = sigma_s . va + sum_j T_sj (vb_j + (sigma V)_sj)
//   w_s  = u_s - ubar,   ubar = Obar . v = mean_s u_s
//   S v  = (1/B) [ sum_s sigma_s w_s | sum_s conj(T_s) w_s |
//                  sum_s sigma_s (x) conj(T_s) w_s ]
// Centering u with ubar (known from Obar . p, a P-dot product of the
// previous phase) makes O^dag w the covariance form directly: no
// cancellation between O^dag u / B and Obar^* ubar, and
//   p^dag (S + lambda I) p = (1/B) sum_s |w_s|^2 + lambda |p|^2
// comes from the walker phase, which saves the grid barrier of a separate
// p . Ap reduction.  The CG is Hestenes-Stiefel from x = 0, optionally with
// the Jacobi preconditioner diag(S) + lambda, stopping at |r| <= tol |F|.
//
// Per CG iteration (three grid barriers):
//   W   walker phase (each CTA its walker range):
//       W1: D1 = sigma V on the tensor cores (A = sigma tile [128 walkers x
//           32 sites] exact in bf16, B = three bf16 planes of V [256 columns
//           (Re/Im of 128 hidden units) x 32 sites], streamed by bulk copies
//           through a 3-stage ring), then u_s from D1 (TMEM) and T (global);
//       W2: D2^T = Y^T sigma on the tensor cores (A = three bf16 planes of
//           Y_sn = (conj(T_sj) w_s).{re,im} [128 columns x 32 walkers],
//           formed by the compute warps, B = sigma^T [sites x 32 walkers]),
//           accumulated over the CTA's walkers, then written as the CTA's
//           partial row; the a- and b-sums on the CUDA cores.
//   |   grid barrier
//   C   each CTA its slice of P: S p from the partial rows (Kahan-compensated
//       float32 sums in a fixed order), alpha, x += alpha p, r -= alpha S p.
//   |   grid barrier
//   P   convergence test; beta; p = z + beta p; the bf16 planes of the new p.
//   |   grid barrier
//
// Warp 0 (one thread) issues the bulk copies and the MMAs; warps 1-8
// ("compute warps") do everything else.  Every wait is bounded: a wait that
// gives up sets CR_ETIMEOUT and a global abort flag, after which all CTAs
// leave the solve at their next grid barrier.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace {

constexpr int FC_THREADS = 288;                 // warp 0 + 8 compute warps
constexpr int NCT = 256;                        // compute threads
constexpr int NS1 = 3;                          // W1 operand stages
constexpr int W1_A = 128 * 32 * 2;              // sigma tile of one K-chunk
constexpr int W1_B_PLANE = 256 * 32 * 2;        // one bf16 plane of V, 256 columns
constexpr int W1_STAGE = W1_A + 3 * W1_B_PLANE; // 56 KB
constexpr int Y_BLK = 128 * 32 * 2;             // one plane of one 128-column n-block
constexpr uint32_t WAIT_LIMIT = 1u << 26;       // mbarrier polls
constexpr unsigned BAR_LIMIT = 1u << 23;        // grid-barrier polls (~1 s with the sleeps)
constexpr int MAX_WPC = 1024;                   // walkers per CTA

struct Geo {
    int N, M, P, B;
    int G;       // CTAs
    int wpc;     // walkers per CTA (the last CTA may have fewer)
    int ntpc;    // W1 walker tiles per CTA
    int trows;   // rows per W1 tile (<= 128)
    int Kp;      // sites padded to a multiple of 32 (W1 contraction length)
    int nkc1;    // W1 K-chunks of 32 sites
    int npass1;  // W1 column passes of 256 (the last one wlast1 wide)
    int wlast1;
    int Np;      // sites padded to a multiple of 16 (W2 MMA N)
    int nb2;     // W2 n-blocks of 128 columns of Y
    int nbp;     // n-blocks per W2 pass (<= 2)
    int npass2;
    int nwc;     // W2 walker chunks of 32 per CTA
    int kslice;  // parameters per CTA in phases C and P
    size_t ring; // bytes of the operand ring (W1 and W2 share it)
    size_t smem; // dynamic shared memory
};

struct Args {
    Geo g;
    const int8_t* spins;
    const cpx<float>* T;
    const cpx<double>* F;
    const cpx<double>* sO;    // sums over walkers: sum O_k [P], then sum |T_j|^2 at P + 2 + j
    double shift, tol;
    int maxit, precond, apply_only;
    const cpx<double>* v_in;  // apply_only: the vector v
    cpx<float>* u_out;        // apply_only: u = O v [B] (or NULL)
    double* cg;               // complex128 x, r, p, Ap, d [5][P]
    unsigned char* a1;        // sigma tiles of W1, per CTA
    unsigned char* b2;        // sigma^T chunks of W2, per CTA
    unsigned char* v2;        // three bf16 planes of the W part of p
    size_t v2_plane;
    cpx<float>* vab;          // float32 a- and b-parts of p [N + M]
    float* part;              // partial rows, complex float32 [G][P]
    double* psc;              // scalar partials [G][8]
    unsigned* bar;            // [0] grid-barrier counter, [1] abort flag
    double* scal;             // [1] F.F, [2] done, [3] iterations, [4] r.r
    int* status;
};

// scalar partial slots
enum { S_WW = 0, S_RR = 1, S_RZ = 2, S_FF = 3, S_OPR = 4, S_OPI = 5, S_PP = 6 };

CR_D void split3(float x, __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo) {
    *hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(*hi);
    *mid = __float2bfloat16_rn(r1);
    *lo = __float2bfloat16_rn(r1 - __bfloat162float(*mid));
}

CR_D __nv_bfloat16 split_term(float x, int pl) {
    __nv_bfloat16 h, m, l;
    split3(x, &h, &m, &l);
    return pl == 0 ? h : (pl == 1 ? m : l);
}

CR_D uint4 pack8(const __nv_bfloat16* v) {
    uint4 r;
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        w[q] = (uint32_t)__bfloat16_as_ushort(v[2 * q]) |
               ((uint32_t)__bfloat16_as_ushort(v[2 * q + 1]) << 16);
    return r;
}

CR_D void kadd(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

CR_D unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// generic-proxy global writes -> visible to later bulk copies (async proxy)
CR_D void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;\n" ::: "memory"); }

// barrier among the 256 compute threads (warps 1-8)
CR_D void compute_sync() { asm volatile("bar.sync 1, 256;\n" ::: "memory"); }

CR_D void mbar_arrive(uint64_t* mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(tc::smem_u32(mbar)) : "memory");
}

// byte offset of element (row, k) in a 32-column K-major tile
CR_D uint32_t koff(int row, int k) { return tc::kmajor_offset(row, k, 32); }

// offset (bytes, within one plane) of element (column n, site i) of the W1
// operand of V: blocks [pass of 256 columns][K-chunk of 32 sites]
CR_HD size_t v2_offset(const Geo& g, int n, int i) {
    const int ps = n >> 8, nl = n & 255, kc = i >> 5, il = i & 31;
    const int width = ps < g.npass1 - 1 ? 256 : g.wlast1;
    return ((size_t)256 * ps * g.Kp + (size_t)width * 32 * kc) * 2 +
           tc::kmajor_offset(nl, il, 32);
}

struct Smem {
    unsigned char* ring;
    cpx<float>* wbuf;   // [wpc] centred u of the CTA's walkers
    cpx<float>* va;     // [N]
    cpx<float>* vb;     // [M]
    cpx<float>* xch;    // [256] exchange
    double* red;        // [64]
    uint64_t* mb;       // mbarriers
    uint32_t* slot;     // TMEM address
    int* flag;          // [0] CTA abort, [1] done
    double* bc;         // [8] broadcast scalars
};

// mbarrier indices
enum { FULL1 = 0, EMPTY1 = 3, D1FULL = 6, D1EMPTY = 8, FULL2 = 10, EMPTY2 = 12, D2FULL = 14, NMB = 15 };

CR_D Smem carve(unsigned char* sm, const Geo& g) {
    Smem s;
    s.ring = sm;
    unsigned char* p = sm + g.ring;
    s.wbuf = (cpx<float>*)p;
    p += (size_t)MAX_WPC * 8;
    s.va = (cpx<float>*)p;
    p += 256 * 8;
    s.vb = (cpx<float>*)p;
    p += 256 * 8;
    s.xch = (cpx<float>*)p;
    p += 256 * 8;
    s.red = (double*)p;
    p += 64 * 8;
    s.bc = (double*)p;
    p += 8 * 8;
    s.mb = (uint64_t*)p;
    p += NMB * 8;
    s.slot = (uint32_t*)p;
    p += 16;
    s.flag = (int*)p;
    return s;
}

// Bounded mbarrier wait; gives up at once after a CTA abort.
CR_D bool wait_mb(uint64_t* mb, uint32_t parity, volatile int* flag, unsigned* bar, int* status) {
    if (flag[0]) return false;
    for (int rep = 0; rep < 64; ++rep) {
        if (tc::mbar_wait(mb, parity, WAIT_LIMIT >> 6)) return true;
        if (flag[0] || *(volatile unsigned*)&bar[1]) {
            flag[0] = 1;
            return false;
        }
    }
    flag[0] = 1;
    atomicExch(&bar[1], 1u);
    set_status(status, CR_ETIMEOUT);
    return false;
}

// Grid barrier (all threads of every CTA): arrive on the counter, wait
// (bounded) until all G CTAs of this round arrived.  Returns false after an
// abort anywhere.
CR_D bool grid_sync(unsigned* bar, unsigned target, volatile int* flag, int* status) {
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&bar[0], 1u);
        unsigned n = 0;
        for (;;) {
            if (ld_acquire(&bar[0]) >= target) break;
            if (*(volatile unsigned*)&bar[1]) {
                flag[0] = 1;
                break;
            }
            if (++n > BAR_LIMIT) {
                flag[0] = 1;
                atomicExch(&bar[1], 1u);
                set_status(status, CR_ETIMEOUT);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
    }
    __syncthreads();
    tc::fence_after_sync();
    return flag[0] == 0;
}

// Sum of v over the 256 compute threads (float64), result in every one.
CR_D double csum(double v, double* red) {
    v = warp_sum(v);
    const int cw = (threadIdx.x >> 5) - 1, lane = threadIdx.x & 31;
    compute_sync();
    if (lane == 0) red[cw] = v;
    compute_sync();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    compute_sync();
    return t;
}

// sum over CTAs of scalar partial slot `sl`, fixed order (identical in every CTA)
CR_D double sum_psc(const double* psc, int G, int sl) {
    const int lane = threadIdx.x & 31;
    double v = 0.0;
    for (int c = lane; c < G; c += 32) v += psc[(size_t)c * 8 + sl];
    return warp_sum(v);
}

// The operands of p_k (value pk) for the walker phase: float32 a/b parts,
// bf16 planes of the W part.  Also accumulates Obar . p and |p|^2.
CR_D void emit_p(const Args& a, int k, cpx<double> pk) {
    const Geo& g = a.g;
    const int N = g.N, M = g.M;
    if (k < N + M) {
        a.vab[k] = ccast<float>(pk);
        return;
    }
    const int i = (k - N - M) / M, j = (k - N - M) % M;
    const float re = (float)pk.x, im = (float)pk.y;
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
        __nv_bfloat16* base = (__nv_bfloat16*)(a.v2 + pl * a.v2_plane);
        base[v2_offset(g, 2 * j, i) / 2] = split_term(re, pl);
        base[v2_offset(g, 2 * j + 1, i) / 2] = split_term(im, pl);
    }
}

}  // namespace

__global__ void __launch_bounds__(FC_THREADS, 1) cg_fused_kernel(const __grid_constant__ Args a) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const Geo& g = a.g;
    const int N = g.N, M = g.M, P = g.P, B = g.B, G = g.G;
    const int c = blockIdx.x, t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ct = t - 32;  // compute-thread index (warps 1-8)
    Smem s = carve(sm_raw, g);
    volatile int* flag = s.flag;
    const int s0 = c * g.wpc, s1 = min(B, s0 + g.wpc), nw = max(0, s1 - s0);
    const int k0 = min(P, c * g.kslice), k1 = min(P, k0 + g.kslice);
    cpx<double>* X = (cpx<double>*)a.cg;
    cpx<double>* Rv = X + P;
    cpx<double>* Pv = X + 2 * P;
    cpx<double>* Ap = X + 3 * P;
    cpx<double>* Dg = X + 4 * P;
    const double invB = 1.0 / B;

    if (t == 0) {
        for (int i = 0; i < NMB; ++i) {
            uint32_t cnt = 1;
            if (i == D1EMPTY || i == D1EMPTY + 1) cnt = NCT;
            if (i == FULL2 || i == FULL2 + 1) cnt = 1 + NCT;
            tc::mbar_init(&s.mb[i], cnt);
        }
        tc::fence_mbar_init();
        flag[0] = 0;
        flag[1] = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(s.slot, 512u);
        tc::tmem_relinquish();
    }

    // ---------------------------------------------------------- prologue
    // the spin operands of this CTA's walkers: W1 sigma tiles and W2 sigma^T
    // chunks (zero outside the walker range and past the last site)
    if (ct >= 0) {
        const int n1 = g.ntpc * g.nkc1 * 128 * 4;
        for (int e = ct; e < n1; e += NCT) {
            const int q8 = e & 3, r = (e >> 2) & 127, blk = e >> 9;
            const int tt = blk / g.nkc1, kc = blk % g.nkc1;
            const int sl = tt * g.trows + r, sw = s0 + sl;
            __nv_bfloat16 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int i = kc * 32 + q8 * 8 + q;
                const bool ok = r < g.trows && sl < nw && i < N;
                v[q] = __float2bfloat16_rn(ok ? (float)a.spins[(size_t)sw * N + i] : 0.f);
            }
            *reinterpret_cast<uint4*>(a.a1 + ((size_t)(c * g.ntpc + tt) * g.nkc1 + kc) * W1_A +
                                      koff(r, q8 * 8)) = pack8(v);
        }
        const int n2 = g.nwc * g.Np * 4;
        for (int e = ct; e < n2; e += NCT) {
            const int q8 = e & 3, i = (e >> 2) % g.Np, wc = (e >> 2) / g.Np;
            __nv_bfloat16 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int sl = wc * 32 + q8 * 8 + q;
                const bool ok = sl < nw && i < N;
                v[q] = __float2bfloat16_rn(ok ? (float)a.spins[(size_t)(s0 + sl) * N + i] : 0.f);
            }
            *reinterpret_cast<uint4*>(a.b2 + ((size_t)c * g.nwc + wc) * g.Np * 64 + koff(i, q8 * 8)) =
                pack8(v);
        }
        // phase P0 on this CTA's slice: x = 0, r = F, z = r / d, p = z
        // (apply_only: p = v), and the operands of p
        double ff = 0.0, rz = 0.0, opr = 0.0, opi = 0.0, pp = 0.0;
        for (int k = k0 + ct; k < k1; k += NCT) {
            cpx<double> pk;
            if (a.apply_only) {
                pk = a.v_in[k];
            } else {
                double d = 1.0;
                if (a.precond) {
                    const double o2 = k < N ? 1.0
                                            : invB * a.sO[P + 2 + (k < N + M ? k - N : (k - N - M) % M)].x;
                    d = o2 - abs2(invB * a.sO[k]) + a.shift;
                }
                const cpx<double> f = a.F[k];
                pk = (1.0 / d) * f;
                X[k] = {0.0, 0.0};
                Rv[k] = f;
                Dg[k] = {d, 0.0};
                ff += abs2(f);
                rz += cmulc(f, pk).x;
            }
            Pv[k] = pk;
            emit_p(a, k, pk);
            const cpx<double> ob = (invB * a.sO[k]) * pk;
            opr += ob.x;
            opi += ob.y;
            pp += abs2(pk);
        }
        fence_proxy_async_global();
        ff = csum(ff, s.red);
        rz = csum(rz, s.red);
        opr = csum(opr, s.red);
        opi = csum(opi, s.red);
        pp = csum(pp, s.red);
        if (ct == 0) {
            double* ps = a.psc + (size_t)c * 8;
            ps[S_FF] = ff;
            ps[S_RZ] = rz;
            ps[S_OPR] = opr;
            ps[S_OPI] = opi;
            ps[S_PP] = pp;
        }
        fence_proxy_async_global();
    }
    unsigned round = 1;
    bool ok = grid_sync(a.bar, round++ * G, flag, a.status);
    const uint32_t taddr = *s.slot;

    // scalars common to all CTAs (warp 1 sums, broadcast through shared memory)
    if (warp == 1) {
        const double ff = sum_psc(a.psc, G, S_FF), rz = sum_psc(a.psc, G, S_RZ);
        if (lane == 0) {
            s.bc[0] = ff;
            s.bc[1] = rz;
        }
    }
    __syncthreads();
    const double ff = s.bc[0];
    double rz = s.bc[1];
    int its = 0, done = (!a.apply_only && ff == 0.0) ? 1 : 0;
    double rr = ff;
    // pipeline counters (identical in every role of the CTA)
    uint32_t g1 = 0, u1 = 0, g2 = 0, u2 = 0;
    // producer only: last copy issued into each stage and last MMA commit, so
    // that an abort can wait (bounded) for what is still in flight
    int last1[NS1] = {-1, -1, -1}, last2[2] = {-1, -1}, lastm1 = -1, lastm2 = -1;

    while (ok && !done && its < (a.apply_only ? 1 : a.maxit)) {
        // ======================================================= walker phase
        if (warp == 1) {
            const double opr = sum_psc(a.psc, G, S_OPR), opi = sum_psc(a.psc, G, S_OPI);
            const double pp = sum_psc(a.psc, G, S_PP);
            if (lane == 0) {
                s.bc[2] = opr;  // ubar = Obar . p
                s.bc[3] = opi;
                s.bc[4] = pp;
            }
        }
        if (ct >= 0) {
            for (int i = ct; i < N; i += NCT) s.va[i] = a.vab[i];
            for (int j = ct; j < M; j += NCT) s.vb[j] = a.vab[N + j];
        }
        __syncthreads();
        const cpx<double> ubar = {s.bc[2], s.bc[3]};
        const cpx<float> ubar32 = ccast<float>(ubar);
        const int units = g.ntpc * g.npass1;
        double ww = 0.0;  // sum |w_s|^2 of this CTA (compute threads)
        if (warp == 0) {
            if (lane == 0) {
                // ----------------------------------------- W1 producer / MMA
                const int total = units * g.nkc1;
                auto width_of = [&](int ps) { return ps < g.npass1 - 1 ? 256 : g.wlast1; };
                auto load = [&](int q) {
                    const uint32_t gq = g1 + q, b = gq % NS1;
                    if (gq >= NS1 && !wait_mb(&s.mb[EMPTY1 + b], ((gq / NS1) - 1) & 1, flag, a.bar, a.status))
                        return;
                    const int unit = q / g.nkc1, kc = q % g.nkc1;
                    const int tt = unit / g.npass1, ps = unit % g.npass1, w = width_of(ps);
                    unsigned char* st = s.ring + (size_t)b * W1_STAGE;
                    tc::mbar_expect_tx(&s.mb[FULL1 + b], (uint32_t)(W1_A + 3 * w * 64));
                    tc::bulk_g2s(st, a.a1 + ((size_t)(c * g.ntpc + tt) * g.nkc1 + kc) * W1_A, W1_A,
                                 &s.mb[FULL1 + b]);
                    const size_t boff = ((size_t)256 * ps * g.Kp + (size_t)w * 32 * kc) * 2;
                    for (int pl = 0; pl < 3; ++pl)
                        tc::bulk_g2s(st + W1_A + pl * W1_B_PLANE, a.v2 + pl * a.v2_plane + boff,
                                     (uint32_t)(w * 64), &s.mb[FULL1 + b]);
                    last1[b] = (int)gq;
                };
                for (int q = 0; q < NS1 - 1 && q < total; ++q) load(q);
                for (int q = 0; q < total; ++q) {
                    if (q + NS1 - 1 < total) load(q + NS1 - 1);
                    const uint32_t gq = g1 + q, b = gq % NS1;
                    const int unit = q / g.nkc1, kc = q % g.nkc1, ps = unit % g.npass1;
                    const uint32_t uu = u1 + unit, h = uu & 1;
                    if (kc == 0 && uu >= 2)
                        wait_mb(&s.mb[D1EMPTY + h], ((uu >> 1) - 1) & 1, flag, a.bar, a.status);
                    wait_mb(&s.mb[FULL1 + b], (gq / NS1) & 1, flag, a.bar, a.status);
                    tc::fence_after_sync();
                    const int w = width_of(ps);
                    const uint32_t idesc = tc::make_idesc_bf16(128, w);
                    const uint32_t sa = tc::smem_u32(s.ring + (size_t)b * W1_STAGE);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
                        for (int pl = 0; pl < 3; ++pl) {
                            const uint64_t ad = tc::make_desc(sa + ks * 256, 128, 512);
                            const uint64_t bd =
                                tc::make_desc(sa + W1_A + pl * W1_B_PLANE + ks * 256, 128, 512);
                            tc::mma_bf16(taddr + 256 * h, ad, bd, idesc, (kc | ks | pl) != 0);
                        }
                    tc::commit(&s.mb[EMPTY1 + b]);
                    lastm1 = (int)gq;
                    if (kc == g.nkc1 - 1) tc::commit(&s.mb[D1FULL + h]);
                }
            }
            __syncwarp();
        } else {
            // --------------------------------------------- W1 compute warps
            const int lb = warp & 3, hf = (warp - 1) >> 2, row = 32 * lb + lane;
            cpx<float> uacc = {0.f, 0.f};
            for (int unit = 0; unit < units; ++unit) {
                const int tt = unit / g.npass1, ps = unit % g.npass1;
                const uint32_t uu = u1 + unit, h = uu & 1;
                const int sl = tt * g.trows + row;
                const bool valid = row < g.trows && sl < nw;
                const int sw = s0 + sl;
                if (ps == 0) {
                    // sigma . va: the two threads of a row take alternate sites
                    uacc = {0.f, 0.f};
                    if (valid)
                        for (int i = hf; i < N; i += 2)
                            uacc = uacc + (float)a.spins[(size_t)sw * N + i] * s.va[i];
                }
                wait_mb(&s.mb[D1FULL + h], (uu >> 1) & 1, flag, a.bar, a.status);
                tc::fence_after_sync();
                const int w = ps < g.npass1 - 1 ? 256 : g.wlast1;
                for (int grp = hf; grp < w / 16; grp += 2) {
                    float d[16];
                    tc::tmem_ld16(taddr + ((uint32_t)(32 * lb) << 16) + 256 * h + 16 * grp, d);
                    const int j0 = 128 * ps + 8 * grp;
                    if (valid) {
                        const cpx<float>* Tr = a.T + (size_t)sw * M;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int j = j0 + q;
                            if (j < M) {
                                const cpx<float> x = {d[2 * q] + s.vb[j].x, d[2 * q + 1] + s.vb[j].y};
                                uacc = uacc + ldg(Tr + j) * x;
                            }
                        }
                    }
                }
                tc::fence_before_sync();
                mbar_arrive(&s.mb[D1EMPTY + h]);
                if (ps == g.npass1 - 1) {
                    // u of the tile's rows: the two column halves meet
                    if (hf == 1) s.xch[row] = uacc;
                    compute_sync();
                    if (hf == 0 && row < g.trows && sl < g.wpc) {
                        cpx<float> wv = {0.f, 0.f};
                        if (valid) {
                            const cpx<float> u = uacc + s.xch[row];
                            if (a.u_out) a.u_out[sw] = u;
                            wv = u - ubar32;
                            ww += (double)abs2(wv);
                        }
                        s.wbuf[sl] = wv;
                    }
                    compute_sync();
                }
            }
            // a-sums: sum_s sigma_si w_s per site (Kahan), into the partial row
            compute_sync();
            for (int i = ct; i < N; i += NCT) {
                float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
                for (int sl = 0; sl < nw; ++sl) {
                    const float sg = (float)a.spins[(size_t)(s0 + sl) * N + i];
                    kadd(sx, cx, sg * s.wbuf[sl].x);
                    kadd(sy, cy, sg * s.wbuf[sl].y);
                }
                a.part[2 * ((size_t)c * P + i)] = sx - cx;
                a.part[2 * ((size_t)c * P + i) + 1] = sy - cy;
            }
        }
        g1 += units * g.nkc1;
        u1 += units;
        // TMEM: every D1 read is done before the W2 MMAs reuse the columns
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();

        for (int ps2 = 0; ps2 < g.npass2; ++ps2) {
            const int nbq = min(g.nbp, g.nb2 - ps2 * g.nbp);
            const int jp0 = 64 * g.nbp * ps2, Jp = 64 * nbq;
            const size_t stage2 = (size_t)g.nbp * 3 * Y_BLK + (size_t)g.Np * 64;
            if (warp == 0) {
                if (lane == 0) {
                    // ------------------------------------ W2 producer / MMA
                    auto load = [&](int wc) {
                        const uint32_t gq = g2 + wc, b = gq & 1;
                        if (gq >= 2 && !wait_mb(&s.mb[EMPTY2 + b], ((gq >> 1) - 1) & 1, flag, a.bar,
                                                a.status))
                            return;
                        unsigned char* st = s.ring + b * stage2 + (size_t)g.nbp * 3 * Y_BLK;
                        tc::mbar_expect_tx(&s.mb[FULL2 + b], (uint32_t)(g.Np * 64));
                        tc::bulk_g2s(st, a.b2 + ((size_t)c * g.nwc + wc) * g.Np * 64,
                                     (uint32_t)(g.Np * 64), &s.mb[FULL2 + b]);
                        last2[b] = (int)gq;
                    };
                    const uint32_t idesc = tc::make_idesc_bf16(128, g.Np);
                    load(0);
                    for (int wc = 0; wc < g.nwc; ++wc) {
                        if (wc + 1 < g.nwc) load(wc + 1);
                        const uint32_t gq = g2 + wc, b = gq & 1;
                        wait_mb(&s.mb[FULL2 + b], (gq >> 1) & 1, flag, a.bar, a.status);
                        tc::fence_after_sync();
                        const uint32_t sy = tc::smem_u32(s.ring + b * stage2);
                        const uint32_t ss = sy + (uint32_t)(g.nbp * 3 * Y_BLK);
                        for (int nb = 0; nb < nbq; ++nb)
#pragma unroll
                            for (int pl = 0; pl < 3; ++pl)
#pragma unroll
                                for (int ks = 0; ks < 2; ++ks) {
                                    const uint64_t ad =
                                        tc::make_desc(sy + (pl * g.nbp + nb) * Y_BLK + ks * 256, 128, 512);
                                    const uint64_t bd = tc::make_desc(ss + ks * 256, 128, 512);
                                    tc::mma_bf16(taddr + nb * g.Np, ad, bd, idesc, (wc | pl | ks) != 0);
                                }
                        tc::commit(&s.mb[EMPTY2 + b]);
                        lastm2 = (int)gq;
                    }
                    tc::commit(&s.mb[D2FULL]);
                }
                __syncwarp();
            } else {
                // ---------------------------------------- W2 compute warps
                const int tpj = NCT / Jp;  // threads per hidden unit: 2 or 4
                const int j = jp0 + ct % Jp;
                float bsx = 0.f, bsy = 0.f, bcx = 0.f, bcy = 0.f;
                for (int wc = 0; wc < g.nwc; ++wc) {
                    const uint32_t gq = g2 + wc, b = gq & 1;
                    if (gq >= 2) wait_mb(&s.mb[EMPTY2 + b], ((gq >> 1) - 1) & 1, flag, a.bar, a.status);
                    tc::fence_after_sync();
                    unsigned char* sy = s.ring + b * stage2;
                    for (int grp = ct / Jp; grp < 4; grp += tpj) {
                        __nv_bfloat16 h[2][8], m[2][8], l[2][8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int sl = wc * 32 + grp * 8 + q;
                            cpx<float> y = {0.f, 0.f};
                            if (sl < nw && j < M) y = conj(ldg(a.T + (size_t)(s0 + sl) * M + j)) * s.wbuf[sl];
                            kadd(bsx, bcx, y.x);
                            kadd(bsy, bcy, y.y);
                            split3(y.x, &h[0][q], &m[0][q], &l[0][q]);
                            split3(y.y, &h[1][q], &m[1][q], &l[1][q]);
                        }
                        const int nl = 2 * (j - jp0), nb = nl >> 7, r0 = nl & 127;
#pragma unroll
                        for (int cmp = 0; cmp < 2; ++cmp) {
                            const uint32_t o = koff(r0 + cmp, grp * 8);
                            *reinterpret_cast<uint4*>(sy + (0 * g.nbp + nb) * Y_BLK + o) = pack8(h[cmp]);
                            *reinterpret_cast<uint4*>(sy + (1 * g.nbp + nb) * Y_BLK + o) = pack8(m[cmp]);
                            *reinterpret_cast<uint4*>(sy + (2 * g.nbp + nb) * Y_BLK + o) = pack8(l[cmp]);
                        }
                    }
                    tc::fence_proxy_async();
                    mbar_arrive(&s.mb[FULL2 + b]);
                }
                // the pass's D2^T rows -> partial row (W part); b-sums
                wait_mb(&s.mb[D2FULL], u2 & 1, flag, a.bar, a.status);
                tc::fence_after_sync();
                const int lb = warp & 3, hf = (warp - 1) >> 2, row = 32 * lb + lane;
                for (int nb = 0; nb < nbq; ++nb) {
                    const int nl = 128 * nb + row, jj = jp0 + (nl >> 1), cmp = nl & 1;
                    for (int grp = hf; grp < g.Np / 16; grp += 2) {
                        float d[16];
                        tc::tmem_ld16(taddr + ((uint32_t)(32 * lb) << 16) + nb * g.Np + 16 * grp, d);
                        if (jj < M)
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const int i = 16 * grp + q;
                                if (i < N) a.part[2 * ((size_t)c * P + N + M + (size_t)i * M + jj) + cmp] = d[q];
                            }
                    }
                }
                s.xch[ct] = {bsx - bcx, bsy - bcy};
                compute_sync();
                if (ct < Jp && j < M) {
                    cpx<float> tot = s.xch[ct];
                    for (int r = 1; r < tpj; ++r) tot = tot + s.xch[ct + r * Jp];
                    a.part[2 * ((size_t)c * P + N + j)] = tot.x;
                    a.part[2 * ((size_t)c * P + N + j) + 1] = tot.y;
                }
                compute_sync();
            }
            g2 += g.nwc;
            u2 += 1;
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        }
        if (ct >= 0) {
            ww = csum(ww, s.red);
            if (ct == 0) a.psc[(size_t)c * 8 + S_WW] = ww;
        }
        ok = grid_sync(a.bar, round++ * G, flag, a.status);
        if (!ok) break;

        // ================================================ phase C (slice)
        if (warp == 1) {
            const double sww = sum_psc(a.psc, G, S_WW);
            if (lane == 0) s.bc[5] = sww;
        }
        __syncthreads();
        const double pAp = s.bc[5] * invB + a.shift * s.bc[4];
        const double alpha = a.apply_only ? 0.0 : rz / pAp;
        double rrp = 0.0, rzp = 0.0;
        if (ct >= 0) {
            const int L = k1 - k0;
            const int tpk = L <= 64 ? 4 : (L <= 128 ? 2 : 1);
            const int cg = ct % tpk, per = NCT / tpk;
            const cpx<double> du = ubar - ccast<double>(ubar32);
            for (int base = 0; base < L; base += per) {
                const int kk = base + ct / tpk, k = k0 + kk;
                double tx = 0.0, ty = 0.0;
                if (kk < L) {
                    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
                    for (int cc = cg; cc < G; cc += tpk) {
                        const float2 v = *reinterpret_cast<const float2*>(a.part + 2 * ((size_t)cc * P + k));
                        kadd(sx, cx, v.x);
                        kadd(sy, cy, v.y);
                    }
                    tx = (double)sx - (double)cx;
                    ty = (double)sy - (double)cy;
                }
                // fixed-order combination of the tpk lanes (bitwise identical in each)
                for (int o = 1; o < tpk; o <<= 1) {
                    tx += __shfl_xor_sync(0xffffffffu, tx, o);
                    ty += __shfl_xor_sync(0xffffffffu, ty, o);
                }
                if (kk < L && cg == 0) {
                    const cpx<double> ob = invB * a.sO[k];
                    const cpx<double> pk = Pv[k];
                    const cpx<double> apk = invB * cpx<double>{tx, ty} - conj(ob) * du + a.shift * pk;
                    if (a.apply_only) {
                        Ap[k] = apk;
                    } else {
                        X[k] = X[k] + alpha * pk;
                        const cpx<double> rk = Rv[k] - alpha * apk;
                        Rv[k] = rk;
                        const double r2 = abs2(rk);
                        rrp += r2;
                        rzp += r2 / Dg[k].x;
                    }
                }
            }
            rrp = csum(rrp, s.red);
            rzp = csum(rzp, s.red);
            if (ct == 0) {
                a.psc[(size_t)c * 8 + S_RR] = rrp;
                a.psc[(size_t)c * 8 + S_RZ] = rzp;
            }
        }
        ++its;
        if (a.apply_only) break;
        ok = grid_sync(a.bar, round++ * G, flag, a.status);
        if (!ok) break;

        // ================================================ phase P (slice)
        if (warp == 1) {
            const double r2 = sum_psc(a.psc, G, S_RR), rzn = sum_psc(a.psc, G, S_RZ);
            if (lane == 0) {
                s.bc[6] = r2;
                s.bc[7] = rzn;
            }
        }
        __syncthreads();
        rr = s.bc[6];
        const double rz_new = s.bc[7];
        done = !(rr > a.tol * a.tol * ff) ? 1 : 0;
        if (done || its >= a.maxit) break;
        const double beta = rz_new / rz;
        rz = rz_new;
        if (ct >= 0) {
            double opr = 0.0, opi = 0.0, pp = 0.0;
            for (int k = k0 + ct; k < k1; k += NCT) {
                const cpx<double> pk = (1.0 / Dg[k].x) * Rv[k] + beta * Pv[k];
                Pv[k] = pk;
                emit_p(a, k, pk);
                const cpx<double> ob = (invB * a.sO[k]) * pk;
                opr += ob.x;
                opi += ob.y;
                pp += abs2(pk);
            }
            fence_proxy_async_global();
            opr = csum(opr, s.red);
            opi = csum(opi, s.red);
            pp = csum(pp, s.red);
            if (ct == 0) {
                double* ps = a.psc + (size_t)c * 8;
                ps[S_OPR] = opr;
                ps[S_OPI] = opi;
                ps[S_PP] = pp;
            }
            fence_proxy_async_global();
        }
        ok = grid_sync(a.bar, round++ * G, flag, a.status);
    }

    if (c == 0 && t == 32 && !a.apply_only) {
        a.scal[1] = ff;
        a.scal[2] = done ? 1.0 : 0.0;
        a.scal[3] = (double)its;
        a.scal[4] = rr;
    }
    // nothing of this CTA is in flight past here on the normal path; after an
    // abort, wait (bounded) for the copies it issued to land and for its last
    // MMA commits, before the shared memory and TMEM are released
    if (flag[0] && t == 0) {
        for (int b = 0; b < NS1; ++b)
            if (last1[b] >= 0) tc::mbar_wait(&s.mb[FULL1 + b], (last1[b] / NS1) & 1, WAIT_LIMIT);
        for (int b = 0; b < 2; ++b)
            if (last2[b] >= 0) tc::mbar_wait(&s.mb[FULL2 + b], (last2[b] >> 1) & 1, WAIT_LIMIT);
        if (lastm1 >= 0)
            tc::mbar_wait(&s.mb[EMPTY1 + lastm1 % NS1], (lastm1 / NS1) & 1, WAIT_LIMIT);
        if (lastm2 >= 0) tc::mbar_wait(&s.mb[EMPTY2 + (lastm2 & 1)], (lastm2 >> 1) & 1, WAIT_LIMIT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512u);
}

// ------------------------------------------------------------------ host

static bool fcg_geometry(const cr_ctx* c, int B, Geo* g) {
    const int N = c->N, M = c->M;
    if (c->prec != CR_MIXED || N > 256 || M > 256 || B < 1) return false;
    g->N = N;
    g->M = M;
    g->P = c->P;
    g->B = B;
    int G = (B + 31) / 32;
    if (G > c->n_sm) G = c->n_sm;
    g->G = G;
    g->wpc = (B + G - 1) / G;
    if (g->wpc > MAX_WPC) return false;
    g->ntpc = (g->wpc + 127) / 128;
    g->trows = (g->wpc + g->ntpc - 1) / g->ntpc;
    g->Kp = ((N + 31) / 32) * 32;
    g->nkc1 = g->Kp / 32;
    const int nc1 = ((2 * M + 15) / 16) * 16;
    g->npass1 = (nc1 + 255) / 256;
    g->wlast1 = nc1 - 256 * (g->npass1 - 1);
    g->Np = ((N + 15) / 16) * 16;
    g->nb2 = (2 * M + 127) / 128;
    g->nbp = g->nb2 < 2 ? g->nb2 : 2;
    g->npass2 = (g->nb2 + g->nbp - 1) / g->nbp;
    g->nwc = (g->wpc + 31) / 32;
    g->kslice = (g->P + G - 1) / G;
    const size_t r1 = (size_t)NS1 * W1_STAGE;
    const size_t r2 = 2 * ((size_t)g->nbp * 3 * Y_BLK + (size_t)g->Np * 64);
    g->ring = r1 > r2 ? r1 : r2;
    g->smem = g->ring + (size_t)MAX_WPC * 8 + 3 * 256 * 8 + 64 * 8 + 8 * 8 + NMB * 8 + 16 + 16;
    return g->smem <= 227 * 1024;
}

// Workspace of the fused solve for up to max_walkers walkers (bytes per
// buffer), or false if the context is not covered.
bool fcg_supported(const cr_ctx* c) {
    Geo g;
    return fcg_geometry(c, c->max_walkers, &g);
}

void fcg_sizes(const cr_ctx* c, size_t* a1, size_t* b2, size_t* v2plane, size_t* part) {
    Geo g;
    fcg_geometry(c, c->max_walkers, &g);
    // the largest tile / chunk counts over walker counts up to max_walkers:
    // every CTA count G <= n_sm with wpc = ceil(B / G) <= ceil(max_walkers / G)
    const int ntpc = (((c->max_walkers + c->n_sm - 1) / c->n_sm) + 127) / 128;
    size_t nt = 0, nc = 0;
    for (int G = 1; G <= c->n_sm; ++G) {
        const int wpc = (c->max_walkers + G - 1) / G;
        if (wpc > MAX_WPC) continue;
        const size_t t1 = (size_t)G * ((wpc + 127) / 128), t2 = (size_t)G * ((wpc + 31) / 32);
        if (t1 > nt) nt = t1;
        if (t2 > nc) nc = t2;
    }
    (void)ntpc;
    *a1 = nt * g.nkc1 * W1_A;
    *b2 = nc * (size_t)g.Np * 64;
    *v2plane = (size_t)256 * g.npass1 * g.Kp * 2;
    *part = (size_t)c->n_sm * c->P * 8;
}

cr_status fcg_prepare(cr_ctx* c) {
    cudaError_t e = cudaFuncSetAttribute(cg_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         227 * 1024);
    return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "fcg_prepare: %s", cudaGetErrorString(e));
}

// One fused solve (apply_only = 0) or one product (S + shift I) v into
// cg[3P] (apply_only = 1).  redO: walker sums of O and |T|^2.
cr_status launch_cg_fused(cr_ctx* c, const int8_t* spins, const void* T, int B, const double* redO,
                          double shift, double tol, int maxit, int precond, int apply_only,
                          const double* v_in, void* u_out) {
    Args a;
    if (!fcg_geometry(c, B, &a.g)) return cr_fail(c, CR_EINVAL, "fused CG: unsupported shape");
    a.spins = spins;
    a.T = (const cpx<float>*)T;
    a.F = (const cpx<double>*)c->F;
    a.sO = (const cpx<double>*)redO;
    a.shift = shift;
    a.tol = tol;
    a.maxit = maxit;
    a.precond = precond;
    a.apply_only = apply_only;
    a.v_in = (const cpx<double>*)v_in;
    a.u_out = (cpx<float>*)u_out;
    a.cg = c->cg;
    a.a1 = c->fcg_a1;
    a.b2 = c->fcg_b2;
    a.v2 = c->fcg_v2;
    a.v2_plane = c->fcg_v2plane;
    a.vab = (cpx<float>*)c->fcg_vab;
    a.part = (float*)c->fcg_part;
    a.psc = c->fcg_psc;
    a.bar = c->fcg_bar;
    a.scal = c->scal;
    a.status = c->d_status;
    cudaError_t e = cudaMemsetAsync(c->fcg_bar, 0, 2 * sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return cr_fail(c, CR_ECUDA, "fused CG: %s", cudaGetErrorString(e));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.g.G);
    cfg.blockDim = dim3(FC_THREADS);
    cfg.dynamicSmemBytes = a.g.smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CR_LAUNCH(c, CR_KERNEL_FCG, e = cudaLaunchKernelEx(&cfg, cg_fused_kernel, a));
    if (e != cudaSuccess) return cr_fail(c, CR_ECUDA, "cg_fused_kernel: %s", cudaGetErrorString(e));
    return cr_check_launch(c, "cg_fused_kernel");
}
