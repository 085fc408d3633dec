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
// The CG is the Chronopoulos-Gear form of Hestenes-Stiefel CG (Chronopoulos
// and Gear, J. Comput. Appl. Math. 25, 1989): with u = M^-1 r and w = A u,
//   gamma = (r, u), delta = (u, A u), beta = gamma / gamma_prev,
//   alpha = gamma / (delta - beta gamma / alpha_prev),
//   p = u + beta p, s = w + beta s (s = A p), x += alpha p, r -= alpha s,
// the same iterates as the textbook recursion in exact arithmetic, with both
// inner products of an iteration formed together: delta comes out of the
// walker phase (the centred form above) and gamma from the slice phase, so
// an iteration needs two grid barriers.  Should the recurrence's (p, A p)
// lose positivity to rounding, the iteration restarts (beta = 0).
//
// Per CG iteration:
//   W   walker phase (each CTA its walker range), the product A u:
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
//   S   each CTA its slice of P: A u from the partial rows (Kahan-compensated
//       float32 sums in a fixed order), alpha, beta, the updates of p, s, x,
//       r, the new u and its bf16 planes, the partial inner products.
//   |   grid barrier
// The convergence test |r| <= tol |F| opens each walker phase; the operand
// copies of that phase start before it, the MMAs after it.
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
constexpr int MAX_WPC = 512;                    // walkers per CTA
constexpr int KS_MAX = 512;                     // parameters per CTA (its CG slice in smem)

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

// scalar partial slots, one value per CTA: psc[cta * 8 + slot]
enum { S_WW = 0, S_RR = 1, S_GAM = 2, S_FF = 3, S_OUR = 4, S_OUI = 5, S_UU = 6 };

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
    // the CTA's slice of the CG vectors, resident for the whole solve
    cpx<double>* x;     // [KS_MAX]
    cpx<double>* r;
    cpx<double>* p;
    cpx<double>* sv;    // s = A p
    cpx<double>* ob;    // Obar_k = (sum_s O_sk) / B
    double* d;          // Jacobi diagonal (1 without preconditioning)
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
enum { FULL1 = 0, EMPTY1 = 3, D1FULL = 6, D1EMPTY = 8, FULL2 = 10, EMPTY2 = 12, D2FULL = 14, GO = 15,
       NMB = 16 };

CR_D Smem carve(unsigned char* sm, const Geo& g) {
    Smem s;
    s.ring = sm;
    unsigned char* p = sm + g.ring;
    s.x = (cpx<double>*)p;
    p += KS_MAX * 16;
    s.r = (cpx<double>*)p;
    p += KS_MAX * 16;
    s.p = (cpx<double>*)p;
    p += KS_MAX * 16;
    s.sv = (cpx<double>*)p;
    p += KS_MAX * 16;
    s.ob = (cpx<double>*)p;
    p += KS_MAX * 16;
    s.d = (double*)p;
    p += KS_MAX * 8;
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
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;\n" ::"l"(&bar[0]) : "memory");
        unsigned n = 0;
        for (;;) {
            if (*(volatile unsigned*)&bar[0] >= target) break;
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
            if (n > 4096) __nanosleep(64);  // spin first: most waits are a few microseconds
        }
        asm volatile("fence.acq_rel.gpu;\n" ::: "memory");  // acquire what the others released
    }
    __syncthreads();
    tc::fence_after_sync();
    return flag[0] == 0;
}

// The CTA's partials of NV scalar slots (compute threads only): warp sums,
// then one barrier, then the eight warp values of each slot added in a
// fixed tree order and written to psc[cta * 8 + slot].
template <int NV>
CR_D void put_psc(double* psc, int cta, const double (&v)[NV], const int (&sl)[NV], double* red) {
    const int cw = (threadIdx.x >> 5) - 1, lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double w = warp_sum(v[q]);
        if (lane == 0) red[cw * 8 + q] = w;
    }
    compute_sync();
    const int ct = threadIdx.x - 32;
    if (ct < NV) {
        const double* r = red + ct;
        const double tot = ((r[0] + r[8]) + (r[16] + r[24])) + ((r[32] + r[40]) + (r[48] + r[56]));
        psc[(size_t)cta * 8 + sl[ct]] = tot;
    }
}

// Sums over all CTAs of NV slots, by one warp, all loads in flight at once,
// in a fixed order (the same values in every lane and every CTA).
template <int NV>
CR_D void sum_psc(const double* psc, int G, const int (&sl)[NV], double (&out)[NV]) {
    const int lane = threadIdx.x & 31;
    double v[NV][5];
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const int cc = lane + 32 * m;
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q][m] = cc < G ? psc[(size_t)cc * 8 + sl[q]] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double x = (v[q][0] + v[q][1]) + (v[q][2] + v[q][3]);
        for (int cc = lane + 160; cc < G; cc += 32) x += psc[(size_t)cc * 8 + sl[q]];
        out[q] = warp_sum(x + v[q][4]);
    }
}

// The operands of entry k (value pk) of the vector the walker phase
// multiplies: float32 a- and b-parts, three bf16 planes of the W part.
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
    volatile int* flag = s.flag;  // [0] CTA abort, [1] solve finished
    const int s0 = c * g.wpc, s1 = min(B, s0 + g.wpc), nw = max(0, s1 - s0);
    const int k0 = min(P, c * g.kslice), k1 = min(P, k0 + g.kslice);
    cpx<double>* X = (cpx<double>*)a.cg;
    cpx<double>* Ap = X + 3 * P;
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
        // this CTA's slice: x = 0, r = F, p = s = 0, u = r / d (apply_only:
        // u = v), the operands of u and the partial inner products
        double ff = 0.0, gam = 0.0, our = 0.0, oui = 0.0, uu = 0.0;
        for (int k = k0 + ct; k < k1; k += NCT) {
            const int kl = k - k0;
            const cpx<double> obk = invB * a.sO[k];
            s.ob[kl] = obk;
            cpx<double> uk;
            if (a.apply_only) {
                uk = a.v_in[k];
                s.r[kl] = uk;
                s.d[kl] = 1.0;
            } else {
                double d = 1.0;
                if (a.precond) {
                    const double o2 = k < N ? 1.0
                                            : invB * a.sO[P + 2 + (k < N + M ? k - N : (k - N - M) % M)].x;
                    d = o2 - abs2(obk) + a.shift;
                }
                const cpx<double> f = a.F[k];
                uk = (1.0 / d) * f;
                s.x[kl] = {0.0, 0.0};
                s.r[kl] = f;
                s.d[kl] = d;
                ff += abs2(f);
                gam += cmulc(f, uk).x;
            }
            s.p[kl] = {0.0, 0.0};
            s.sv[kl] = {0.0, 0.0};
            emit_p(a, k, uk);
            const cpx<double> ou = obk * uk;
            our += ou.x;
            oui += ou.y;
            uu += abs2(uk);
        }
        fence_proxy_async_global();
        const double pv[6] = {ff, ff, gam, our, oui, uu};
        const int ps[6] = {S_FF, S_RR, S_GAM, S_OUR, S_OUI, S_UU};
        put_psc<6>(a.psc, c, pv, ps, s.red);
    }
    unsigned round = 1;
    bool ok = grid_sync(a.bar, round++ * G, flag, a.status);
    const uint32_t taddr = *s.slot;

    int its = 0, done = 0;
    double ff = 0.0, rr = 0.0, gam = 0.0, gam_prev = 1.0, alpha_prev = 1.0;
    // pipeline counters (identical in every role of the CTA)
    uint32_t g1 = 0, u1 = 0, g2 = 0, u2 = 0;
    // producer only: last copy issued into each stage and last MMA commit, so
    // that an abort can wait (bounded) for what is still in flight
    int last1[NS1] = {-1, -1, -1}, last2[2] = {-1, -1}, lastm1 = -1, lastm2 = -1;
    const int units = g.ntpc * g.npass1;
    const int total1 = units * g.nkc1;
    auto width_of = [&](int ps) { return ps < g.npass1 - 1 ? 256 : g.wlast1; };

    while (ok) {
        // ======================================================= walker phase
        // producer: W1 operand copies start at once (their data was released
        // before the barrier); the MMAs wait for the convergence decision
        auto load1 = [&](int q) {
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
        const int npre = NS1 - 1 < total1 ? NS1 - 1 : total1;
        if (t == 0)
            for (int q = 0; q < npre; ++q) load1(q);
        if (warp == 1) {
            // the inner products of the current r and u, and the decision
            const int sl6[6] = {S_RR, S_GAM, S_OUR, S_OUI, S_UU, S_FF};
            double v6[6];
            sum_psc<6>(a.psc, G, sl6, v6);
            const double r2 = v6[0], gm = v6[1], our = v6[2], oui = v6[3], uu = v6[4], f2 = v6[5];
            if (lane == 0) {
                if (its == 0) s.bc[0] = f2;
                const double fnorm2 = s.bc[0];
                const int conv = !a.apply_only && !(r2 > a.tol * a.tol * fnorm2);
                // the decision of the whole CTA: converged, out of iterations, or aborted
                const int fin = conv || (!a.apply_only && its >= a.maxit) || flag[0];
                s.bc[7] = conv;
                s.bc[1] = r2;
                s.bc[2] = our;  // ubar = Obar . u
                s.bc[3] = oui;
                s.bc[4] = uu;
                s.bc[6] = gm;
                flag[1] = fin;
                mbar_arrive(&s.mb[GO]);
            }
        }
        if (ct >= 0) {
            for (int i = ct; i < N; i += NCT) s.va[i] = a.vab[i];
            for (int j = ct; j < M; j += NCT) s.vb[j] = a.vab[N + j];
        }
        // the decision reaches warp 0 through GO, the compute warps through
        // their barrier; flag[1], written once before either, is uniform
        if (warp == 0) wait_mb(&s.mb[GO], (uint32_t)its & 1, flag, a.bar, a.status);
        if (ct >= 0) compute_sync();
        ff = s.bc[0];
        rr = s.bc[1];
        gam = s.bc[6];
        if (flag[1]) {
            // finished: let the copies issued above land, then leave
            if (t == 0)
                for (int q = 0; q < npre; ++q) {
                    const uint32_t gq = g1 + q;
                    tc::mbar_wait(&s.mb[FULL1 + gq % NS1], (gq / NS1) & 1, WAIT_LIMIT);
                }
            done = s.bc[7] != 0.0;
            __syncthreads();
            break;
        }
        const cpx<double> ubar = {s.bc[2], s.bc[3]};
        const cpx<float> ubar32 = ccast<float>(ubar);
        const double uu = s.bc[4];
        double ww = 0.0;  // sum |w_s|^2 of this thread's walkers
        if (warp == 0) {
            if (lane == 0) {
                // ----------------------------------------- W1 producer / MMA
                for (int q = 0; q < total1; ++q) {
                    if (q + NS1 - 1 < total1 && q + NS1 - 1 >= npre) load1(q + NS1 - 1);
                    const uint32_t gq = g1 + q, b = gq % NS1;
                    const int unit = q / g.nkc1, kc = q % g.nkc1, ps = unit % g.npass1;
                    const uint32_t uu1 = u1 + unit, h = uu1 & 1;
                    if (kc == 0 && uu1 >= 2)
                        wait_mb(&s.mb[D1EMPTY + h], ((uu1 >> 1) - 1) & 1, flag, a.bar, a.status);
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
            const bool vecT = (M & 1) == 0;
            cpx<float> uacc = {0.f, 0.f};
            for (int unit = 0; unit < units; ++unit) {
                const int tt = unit / g.npass1, ps = unit % g.npass1;
                const uint32_t uu1 = u1 + unit, h = uu1 & 1;
                const int sl = tt * g.trows + row;
                const bool valid = row < g.trows && sl < nw;
                const int sw = s0 + sl;
                const cpx<float>* Tr = a.T + (size_t)sw * M;
                const int w = width_of(ps), ngr = w / 16;
                // T of a 16-column group (8 hidden units) as four 16-byte
                // loads, fetched two groups ahead of its use
                auto fetchT = [&](int grp, float4* tv) {
                    const int j0 = 128 * ps + 8 * grp;
                    if (grp >= ngr || !valid) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) tv[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                    } else if (vecT && j0 + 8 <= M) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            tv[q] = __ldg(reinterpret_cast<const float4*>(Tr + j0) + q);
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int j = j0 + 2 * q;
                            const cpx<float> t0 = j < M ? ldg(Tr + j) : cpx<float>{0.f, 0.f};
                            const cpx<float> t1 = j + 1 < M ? ldg(Tr + j + 1) : cpx<float>{0.f, 0.f};
                            tv[q] = make_float4(t0.x, t0.y, t1.x, t1.y);
                        }
                    }
                };
                float4 tc0[4], tc1[4], tc2[4];
                fetchT(hf, tc0);
                fetchT(hf + 2, tc1);
                if (ps == 0) {
                    // sigma . va: the two threads of a row take alternate
                    // 16-site blocks of the row (16-byte loads when N % 16 == 0)
                    uacc = {0.f, 0.f};
                    if (valid) {
                        const int8_t* sr = a.spins + (size_t)sw * N;
                        if ((N & 15) == 0) {
                            for (int b16 = hf; b16 < N / 16; b16 += 2) {
                                const int4 raw = __ldg(reinterpret_cast<const int4*>(sr) + b16);
                                const int8_t* sv = reinterpret_cast<const int8_t*>(&raw);
#pragma unroll
                                for (int q = 0; q < 16; ++q)
                                    uacc = uacc + (float)sv[q] * s.va[16 * b16 + q];
                            }
                        } else {
                            for (int i = hf; i < N; i += 2) uacc = uacc + (float)sr[i] * s.va[i];
                        }
                    }
                }
                wait_mb(&s.mb[D1FULL + h], (uu1 >> 1) & 1, flag, a.bar, a.status);
                tc::fence_after_sync();
                for (int grp = hf; grp < ngr; grp += 2) {
                    fetchT(grp + 4, tc2);
                    float d[16];
                    tc::tmem_ld16(taddr + ((uint32_t)(32 * lb) << 16) + 256 * h + 16 * grp, d);
                    const int j0 = 128 * ps + 8 * grp;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int j = j0 + q;
                        const int jv = j < M ? j : 0;
                        const float4 tq = tc0[q >> 1];
                        const cpx<float> tj = (q & 1) ? cpx<float>{tq.z, tq.w} : cpx<float>{tq.x, tq.y};
                        const cpx<float> x = {d[2 * q] + s.vb[jv].x, d[2 * q + 1] + s.vb[jv].y};
                        uacc = uacc + tj * x;  // tj = 0 past M and on invalid rows
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        tc0[q] = tc1[q];
                        tc1[q] = tc2[q];
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
        }
        g1 += total1;
        u1 += units;
        // TMEM: every D1 read is done before the W2 MMAs reuse the columns
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();

        // a-sums: sum_s sigma_si w_s per site.  Thread (block b16 of 16 sites,
        // walker subset sub) sums its walkers from 16-byte spin loads, eight
        // walkers' loads in flight; each site's nsub partial sums are then
        // added in a fixed order, through the operand ring (idle here).
        if (ct >= 0) {
            const int NG = (N + 15) / 16, nsub = NCT / NG;
            const int b16 = ct % NG, sub = ct / NG;
            cpx<float>* xa = (cpx<float>*)s.ring;  // [nsub][NG * 16]
            if (sub < nsub) {
                float ax[16], ay[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) ax[q] = ay[q] = 0.f;
                for (int sl0 = sub; sl0 < nw; sl0 += 8 * nsub) {
                    int4 raw[8];
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const int sl = sl0 + m * nsub;
                        const int8_t* sr = a.spins + (size_t)(s0 + (sl < nw ? sl : 0)) * N;
                        if (sl >= nw) {
                            raw[m] = make_int4(0, 0, 0, 0);
                        } else if ((N & 15) == 0) {
                            raw[m] = __ldg(reinterpret_cast<const int4*>(sr) + b16);
                        } else {
                            int8_t sv[16];
#pragma unroll
                            for (int q = 0; q < 16; ++q) sv[q] = 16 * b16 + q < N ? sr[16 * b16 + q] : (int8_t)0;
                            memcpy(&raw[m], sv, 16);
                        }
                    }
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const int sl = sl0 + m * nsub;
                        const cpx<float> wv = sl < nw ? s.wbuf[sl] : cpx<float>{0.f, 0.f};
                        const int8_t* sv = reinterpret_cast<const int8_t*>(&raw[m]);
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            ax[q] = fmaf((float)sv[q], wv.x, ax[q]);
                            ay[q] = fmaf((float)sv[q], wv.y, ay[q]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) xa[sub * NG * 16 + 16 * b16 + q] = {ax[q], ay[q]};
            }
            compute_sync();
            for (int i = ct; i < N; i += NCT) {
                float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
                for (int r = 0; r < nsub; ++r) {
                    const cpx<float> v = xa[r * NG * 16 + i];
                    kadd(sx, cx, v.x);
                    kadd(sy, cy, v.y);
                }
                a.part[2 * ((size_t)c * P + i)] = sx - cx;
                a.part[2 * ((size_t)c * P + i) + 1] = sy - cy;
            }
        }
        tc::fence_before_sync();
        __syncthreads();  // the ring is W2's from here
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
                const int ng = 4 / tpj;    // walker groups of 8 per thread and chunk (1 or 2)
                float bsx = 0.f, bsy = 0.f, bcx = 0.f, bcy = 0.f;
                // T of this thread's walkers of a chunk, fetched one chunk ahead
                // (compile-time indices throughout, so the buffers stay in registers)
                cpx<float> tcur[2][8], tnxt[2][8];
#define FCG_FETCH_T(WC, TV)                                                                       \
    _Pragma("unroll") for (int gi = 0; gi < 2; ++gi) {                                            \
        const int grp = ct / Jp + gi * tpj;                                                       \
        _Pragma("unroll") for (int q = 0; q < 8; ++q) {                                           \
            const int sl = (WC) * 32 + grp * 8 + q;                                               \
            TV[gi][q] = (gi < ng && sl < nw && j < M) ? ldg(a.T + (size_t)(s0 + sl) * M + j)       \
                                                      : cpx<float>{0.f, 0.f};                     \
        }                                                                                         \
    }
                FCG_FETCH_T(0, tcur)
                for (int wc = 0; wc < g.nwc; ++wc) {
                    const uint32_t gq = g2 + wc, b = gq & 1;
                    if (wc + 1 < g.nwc) {
                        FCG_FETCH_T(wc + 1, tnxt)
                    }
                    if (gq >= 2) wait_mb(&s.mb[EMPTY2 + b], ((gq >> 1) - 1) & 1, flag, a.bar, a.status);
                    tc::fence_after_sync();
                    unsigned char* sy = s.ring + b * stage2;
#pragma unroll
                    for (int gi = 0; gi < 2; ++gi) {
                        if (gi >= ng) break;
                        const int grp = ct / Jp + gi * tpj;
                        __nv_bfloat16 h[2][8], m[2][8], l[2][8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int sl = wc * 32 + grp * 8 + q;
                            // walkers past the CTA's range contribute exact zeros (their
                            // slots of wbuf are never written)
                            const cpx<float> y = sl < nw ? conj(tcur[gi][q]) * s.wbuf[sl] : cpx<float>{0.f, 0.f};
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
#pragma unroll
                    for (int gi = 0; gi < 2; ++gi)
#pragma unroll
                        for (int q = 0; q < 8; ++q) tcur[gi][q] = tnxt[gi][q];
                }
#undef FCG_FETCH_T
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
            const double pv[1] = {ww};
            const int ps[1] = {S_WW};
            put_psc<1>(a.psc, c, pv, ps, s.red);
        }
        ok = grid_sync(a.bar, round++ * G, flag, a.status);
        if (!ok) break;

        // ================================================= slice phase
        if (warp == 1) {
            const int sl1[1] = {S_WW};
            double v1[1];
            sum_psc<1>(a.psc, G, sl1, v1);
            if (lane == 0) s.bc[5] = v1[0];
        }
        __syncthreads();
        // delta = (u, A u) = (1/B) sum_s |w_s|^2 + lambda |u|^2
        const double delta = s.bc[5] * invB + a.shift * uu;
        // (p, A p) by the recurrence, delta - beta^2 (p_prev, A p_prev); it holds
        // while the directions stay A-conjugate.  When rounding has eroded that
        // (float32-accurate products at a large condition number) it can come
        // out tiny or negative: then the recurrence restarts with beta = 0
        // (p = u, s = A u, a steepest-descent step, whose denominator delta
        // is a sum of squares).
        const double beta0 = its == 0 ? 0.0 : gam / gam_prev;
        const double den = its == 0 ? delta : delta - beta0 * gam / alpha_prev;
        const bool restart = its == 0 || !(den > 1e-6 * delta);
        const double beta = restart ? 0.0 : beta0;
        const double alpha = gam / (restart ? delta : den);
        if (ct >= 0) {
            double r2 = 0.0, gm = 0.0, our = 0.0, oui = 0.0, u2s = 0.0;
            const int L = k1 - k0;
            const int tpk = L <= 64 ? 4 : (L <= 128 ? 2 : 1);
            const int cg = ct % tpk, per = NCT / tpk;
            const cpx<double> du = ubar - ccast<double>(ubar32);
            constexpr int BATCH = 40;
            for (int base = 0; base < L; base += per) {
                const int kk = base + ct / tpk, k = k0 + kk;
                double tx = 0.0, ty = 0.0;
                if (kk < L) {
                    float sx = 0.f, sy = 0.f, cx = 0.f, cy = 0.f;
                    // rows cg, cg + tpk, ... with BATCH loads in flight
                    for (int cb = cg; cb < G; cb += BATCH * tpk) {
                        float2 v[BATCH];
#pragma unroll
                        for (int q = 0; q < BATCH; ++q) {
                            const int cc = cb + q * tpk;
                            v[q] = cc < G ? *reinterpret_cast<const float2*>(a.part + 2 * ((size_t)cc * P + k))
                                          : make_float2(0.f, 0.f);
                        }
#pragma unroll
                        for (int q = 0; q < BATCH; ++q) {
                            kadd(sx, cx, v[q].x);
                            kadd(sy, cy, v[q].y);
                        }
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
                    const cpx<double> uk = (1.0 / s.d[kk]) * s.r[kk];
                    // (A u)_k = (S + lambda) u: the centred O^dag w with the
                    // rounding of ubar put back
                    const cpx<double> auk =
                        invB * cpx<double>{tx, ty} - conj(s.ob[kk]) * du + a.shift * uk;
                    if (a.apply_only) {
                        Ap[k] = auk;
                    } else {
                        const cpx<double> pk = uk + beta * s.p[kk];
                        const cpx<double> sk = auk + beta * s.sv[kk];
                        s.p[kk] = pk;
                        s.sv[kk] = sk;
                        s.x[kk] = s.x[kk] + alpha * pk;
                        const cpx<double> rk = s.r[kk] - alpha * sk;
                        s.r[kk] = rk;
                        const cpx<double> un = (1.0 / s.d[kk]) * rk;
                        emit_p(a, k, un);
                        r2 += abs2(rk);
                        gm += cmulc(rk, un).x;
                        const cpx<double> ou = s.ob[kk] * un;
                        our += ou.x;
                        oui += ou.y;
                        u2s += abs2(un);
                    }
                }
            }
            if (!a.apply_only) {
                fence_proxy_async_global();
                const double pv[5] = {r2, gm, our, oui, u2s};
                const int ps[5] = {S_RR, S_GAM, S_OUR, S_OUI, S_UU};
                put_psc<5>(a.psc, c, pv, ps, s.red);
            }
        }
        gam_prev = gam;
        alpha_prev = alpha;
        ++its;
        if (a.apply_only) break;
        ok = grid_sync(a.bar, round++ * G, flag, a.status);
    }

    if (!a.apply_only && ct >= 0)
        for (int k = k0 + ct; k < k1; k += NCT) X[k] = s.x[k - k0];
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
    if (c->fcg_ctas > 0 && c->fcg_ctas < G) G = c->fcg_ctas;  // the walker-block shape chosen
    const int Gp = (c->P + KS_MAX - 1) / KS_MAX;  // every CTA's CG slice fits in shared memory
    const int Gw = (B + MAX_WPC - 1) / MAX_WPC;   // and its walkers
    if (G < Gp) G = Gp;
    if (G < Gw) G = Gw;
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
    if (g->kslice > KS_MAX) return false;
    const size_t r1 = (size_t)NS1 * W1_STAGE;
    const size_t r2 = 2 * ((size_t)g->nbp * 3 * Y_BLK + (size_t)g->Np * 64);
    g->ring = r1 > r2 ? r1 : r2;
    g->smem = g->ring + (size_t)KS_MAX * 88 + (size_t)MAX_WPC * 8 + 3 * 256 * 8 + 64 * 8 + 8 * 8 +
              NMB * 8 + 16 + 16;
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
