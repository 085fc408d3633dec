// Tensor-core (tcgen05) contractions of the matrix-free natural-gradient solve
// for CR_MIXED contexts (Sec. III: S v = O^dag (O v) / B - ...).
//
// Both products have one operand equal to the spins, sigma = +-1, which bf16
// holds exactly.  The other (float32) operand x is split into three bf16
// terms, hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid) (the
// split of Henry, Tang and Heinecke, "Leveraging the bfloat16 artificial
// intelligence datatype for higher-precision computations", ARITH 2019), so
// sigma * (hi + mid + lo) is formed from exact products with float32
// accumulation in TMEM: about 24 significant bits, like the float32 path.
//
//   ov_tc_kernel      u_s = sum_i sigma_si v_a_i + sum_j T_sj (v_b_j + (sigma V)_sj)
//   oreduce_tc_kernel sum over a walker chunk of sigma_si conj(T_sj) g_s, plus
//                     the a-, b- and scalar sums of oreduce_kernel's partial rows
//
// The explicit S of the Cholesky path (sgram_tc_kernel, further down) has
// float32 values in both operands; both are split (see there).
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace {

constexpr uint32_t WAIT_LIMIT = 1u << 26;  // bounded mbarrier polls

CR_D void split3(float x, __nv_bfloat16* hi, __nv_bfloat16* mid, __nv_bfloat16* lo) {
    *hi = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(*hi);
    *mid = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(*mid);
    *lo = __float2bfloat16_rn(r2);
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

}  // namespace

// ------------------------------------------------------------------ O v
//
// 256 threads.  Shared memory: Bs [NT][3][NCp x Kp] (V_W split, column
// n = 2 j + re/im, K = sites), As [128 x Kp] (spins of one 128-walker tile),
// Ts [2][128 x (TJC + 1)] (T of the tile, TJC complex columns at a time,
// double-buffered, padded rows), vb [M], va [N], part [2][128], one mbarrier
// and the TMEM slot.  A CTA loops over walker tiles; D = sigma V of a tile
// occupies TMEM columns [256 nt, 256 nt + NCp).  Warps w and w + 4 read the
// same TMEM lanes (rows), each half of every TJC-column chunk.
constexpr int OV_THREADS = 256;
constexpr int TJC = 32;  // complex columns of T per staged chunk

__global__ void __launch_bounds__(OV_THREADS, 1) ov_tc_kernel(
    const cpx<float>* __restrict__ v, const int8_t* __restrict__ spins,
    const cpx<float>* __restrict__ T, int B, int N, int M, int Kp, int NCp, int NT,
    int tmem_cols, cpx<float>* __restrict__ u, const double* __restrict__ skip,
    int* __restrict__ status) {
    if (skip && *skip != 0.0) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    const size_t bsz = (size_t)NCp * Kp * 2;
    unsigned char* Bs = sm;
    unsigned char* As = sm + (size_t)NT * 3 * bsz;
    cpx<float>* Ts = (cpx<float>*)(As + (size_t)128 * Kp * 2);       // [2][128][TJC + 1]
    cpx<float>* vb = Ts + 2 * 128 * (TJC + 1);
    cpx<float>* va = vb + M;
    cpx<float>* part = va + N;                                         // [2][128]
    uint64_t* mbar = (uint64_t*)(((uintptr_t)(part + 256) + 15) & ~(uintptr_t)15);
    uint32_t* slot = (uint32_t*)(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, (uint32_t)tmem_cols);
        tc::tmem_relinquish();
    }
    const int kc_n = Kp / 8;
    for (int e = t; e < NT * NCp * kc_n; e += OV_THREADS) {
        const int nt = e / (NCp * kc_n), rem = e % (NCp * kc_n), c = rem / kc_n, kc = rem % kc_n;
        const int j = nt * 128 + (c >> 1);
        __nv_bfloat16 h[8], m[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kc * 8 + q;
            float x = 0.f;
            if (j < M && k < N) {
                cpx<float> w = v[N + M + (size_t)k * M + j];
                x = (c & 1) ? w.y : w.x;
            }
            split3(x, &h[q], &m[q], &l[q]);
        }
        const uint32_t off = tc::kmajor_offset(c, kc * 8, Kp);
        unsigned char* base = Bs + (size_t)nt * 3 * bsz;
        *reinterpret_cast<uint4*>(base + off) = pack8(h);
        *reinterpret_cast<uint4*>(base + bsz + off) = pack8(m);
        *reinterpret_cast<uint4*>(base + 2 * bsz + off) = pack8(l);
    }
    for (int j = t; j < M; j += OV_THREADS) vb[j] = v[N + j];
    for (int i = t; i < N; i += OV_THREADS) va[i] = v[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;
    const uint32_t idesc = tc::make_idesc_bf16(128, NCp);
    const int ntiles = (B + 127) / 128;
    const int nchunk = (M + TJC - 1) / TJC;
    const bool vec16 = (N % 16) == 0;
    const int lb = warp & 3, half = warp >> 2;   // TMEM lane block, column half
    const int row = 32 * lb + lane;
    bool ok = true;
    int it = 0;
    // T chunk ch of tile w0 into buffer b: consecutive threads take consecutive columns
    auto load_T = [&](int w0, int ch, int b) {
        cpx<float>* dst = Ts + (size_t)b * 128 * (TJC + 1);
        for (int e = t; e < 128 * TJC; e += OV_THREADS) {
            const int r = e / TJC, jj = e % TJC, w = w0 + r, j = ch * TJC + jj;
            dst[r * (TJC + 1) + jj] = (w < B && j < M) ? T[(size_t)w * M + j] : cpx<float>{0.f, 0.f};
        }
    };
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int w0 = tile * 128;
        // spins of the tile: two threads per walker, each half of the sites
        {
            const int r = t >> 1, hh = t & 1, w = w0 + r;
            cpx<float> ua = {0.f, 0.f};
            for (int kc = hh * (kc_n / 2); kc < (hh + 1) * (kc_n / 2) + (hh ? kc_n % 2 : 0); ++kc) {
                int8_t sv[8];
                if (vec16 && w < B && kc * 8 + 8 <= N) {
                    uint2 raw = *reinterpret_cast<const uint2*>(spins + (size_t)w * N + kc * 8);
                    memcpy(sv, &raw, 8);
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int k = kc * 8 + q;
                        sv[q] = (w < B && k < N) ? spins[(size_t)w * N + k] : (int8_t)0;
                    }
                }
                __nv_bfloat16 s8[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    s8[q] = __float2bfloat16_rn((float)sv[q]);
                    if (sv[q]) ua = ua + (float)sv[q] * va[kc * 8 + q];
                }
                *reinterpret_cast<uint4*>(As + tc::kmajor_offset(r, kc * 8, Kp)) = pack8(s8);
            }
            ua.x += __shfl_xor_sync(0xffffffffu, ua.x, 1);
            ua.y += __shfl_xor_sync(0xffffffffu, ua.y, 1);
            if (hh == 0) part[r] = ua;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();  // As written; the previous tile's TMEM and Ts reads are done
        tc::fence_after_sync();
        if (t == 0) {
            for (int nt = 0; nt < NT; ++nt)
                for (int sp = 0; sp < 3; ++sp)
                    for (int ks = 0; ks < Kp / 16; ++ks) {
                        const uint64_t ad = tc::make_desc(tc::smem_u32(As) + ks * 256, 128, 16 * Kp);
                        const uint64_t bd = tc::make_desc(
                            tc::smem_u32(Bs + ((size_t)nt * 3 + sp) * bsz) + ks * 256, 128, 16 * Kp);
                        tc::mma_bf16(taddr + nt * 256, ad, bd, idesc, (sp | ks) != 0);
                    }
            tc::commit(mbar);
        }
        load_T(w0, 0, 0);  // overlaps the MMA
        ok = tc::mbar_wait(mbar, it & 1, WAIT_LIMIT) && ok;
        tc::fence_after_sync();
        cpx<float> acc = {0.f, 0.f};
        for (int ch = 0; ch < nchunk; ++ch) {
            __syncthreads();  // chunk ch staged; buffer (ch + 1) & 1 free
            if (ch + 1 < nchunk) load_T(w0, ch + 1, (ch + 1) & 1);
            const cpx<float>* tr = Ts + (size_t)(ch & 1) * 128 * (TJC + 1) + row * (TJC + 1);
            // this warp's half of the chunk: TJC / 2 complex = TJC fp32 columns
            const int j_first = ch * TJC + half * (TJC / 2);
            const int col0 = (j_first / 128) * 256 + 2 * (j_first % 128);
#pragma unroll
            for (int g = 0; g < TJC / 16; ++g) {
                float d[16];
                tc::tmem_ld16(taddr + ((uint32_t)(32 * lb) << 16) + col0 + 16 * g, d);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int jj = half * (TJC / 2) + 8 * g + q, j = ch * TJC + jj;
                    if (j < M) {
                        cpx<float> x = {d[2 * q] + vb[j].x, d[2 * q + 1] + vb[j].y};
                        acc = acc + tr[jj] * x;
                    }
                }
            }
        }
        if (half == 1) part[128 + row] = acc;
        __syncthreads();
        if (half == 0 && w0 + row < B) u[w0 + row] = part[row] + acc + part[128 + row];
        __syncthreads();  // part[] and Ts are rewritten by the next tile
    }
    if (!ok && t == 0) set_status(status, CR_ETIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)tmem_cols);
}

// ------------------------------------------------------- O^dag g reduction
//
// 256 threads; one CTA per (walker chunk, tile of 128 sites).  Per stage of
// KC = 32 walkers, buffer b = stage & 1: As[b] [128 x 32] = sigma^T (sites x
// walkers), Bs[b] [NT][3][NCp x 32] = the bf16 terms of Y^T, Y_sj =
// conj(T_sj) g_s.  D accumulates over the chunk in TMEM; the MMAs of stage s
// run while stage s + 1 is staged into the other buffer.
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS, 1) oreduce_tc_kernel(
    const int8_t* __restrict__ spins, const cpx<float>* __restrict__ T,
    const cpx<float>* __restrict__ g, int B, int N, int M, int P, int chunk, int NCp, int NT,
    int tmem_cols, double* __restrict__ partial, const double* __restrict__ skip,
    int* __restrict__ status) {
    if (skip && *skip != 0.0) return;
    constexpr int KC = 32, HK = 16;  // walkers per stage, per thread half
    extern __shared__ __align__(1024) unsigned char sm[];
    const size_t bsz = (size_t)NCp * KC * 2;
    const size_t stage_bytes = (size_t)NT * 3 * bsz + 128 * KC * 2;
    cpx<float>* gs = (cpx<float>*)(sm + 2 * stage_bytes);               // [2][KC]
    cpx<float>* red = gs + 2 * KC;                                       // [2][128] x 2
    uint64_t* mbar = (uint64_t*)(red + 4 * 128);                        // [2]
    uint32_t* slot = (uint32_t*)(mbar + 2);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int c = blockIdx.x, i0 = blockIdx.y * 128;
    const int s0 = c * chunk, s1 = min(B, s0 + chunk);
    const int r = t & 127, hh = t >> 7;   // site row / column, walker half
    if (t == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, (uint32_t)tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;
    const uint32_t idesc = tc::make_idesc_bf16(128, NCp);
    cpx<float> acca = {0.f, 0.f}, accg = {0.f, 0.f};
    float accgg = 0.f;
    cpx<float> accb[2] = {{0.f, 0.f}, {0.f, 0.f}};
    bool ok = true;
    const int i = i0 + r;
    const int nstage = (s1 - s0 + KC - 1) / KC;
    // register prefetch of one stage: HK spins of site i, HK x NT values of T
    int8_t sp[HK];
    cpx<float> tp[2][HK];
    auto fetch = [&](int sb) {
#pragma unroll
        for (int q = 0; q < HK; ++q) {
            const int s = sb + hh * HK + q;
            sp[q] = (s < s1 && i < N) ? spins[(size_t)s * N + i] : (int8_t)0;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int j = nt * 128 + r;
                tp[nt][q] = (nt < NT && s < s1 && j < M) ? T[(size_t)s * M + j]
                                                         : cpx<float>{0.f, 0.f};
            }
        }
    };
    fetch(s0);
    for (int stage = 0; stage < nstage; ++stage) {
        const int sb = s0 + stage * KC, b = stage & 1;
        unsigned char* Bs = sm + b * stage_bytes;
        unsigned char* As = Bs + (size_t)NT * 3 * bsz;
        cpx<float>* gsb = gs + b * KC;
        // buffer b was read by the MMAs of stage - 2
        if (stage >= 2) {
            ok = tc::mbar_wait(&mbar[b], ((stage - 2) >> 1) & 1, WAIT_LIMIT) && ok;
            tc::fence_after_sync();
        }
        if (t < KC) {
            const int s = sb + t;
            gsb[t] = s < s1 ? g[s] : cpx<float>{0.f, 0.f};
        }
        __syncthreads();
        // sigma^T row r (site i), walkers [hh HK, hh HK + HK)
#pragma unroll
        for (int kc = 0; kc < HK / 8; ++kc) {
            __nv_bfloat16 s8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int qq = kc * 8 + q;
                s8[q] = __float2bfloat16_rn((float)sp[qq]);
                if (sp[qq]) acca = acca + (float)sp[qq] * gsb[hh * HK + qq];
            }
            *reinterpret_cast<uint4*>(As + tc::kmajor_offset(r, hh * HK + kc * 8, KC)) = pack8(s8);
        }
        // Y^T column j = 128 nt + r (real columns 2r, 2r + 1 of n-tile nt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            if (nt >= NT || 2 * r >= NCp) break;  // columns past NCp do not exist in this tile
            unsigned char* base = Bs + (size_t)nt * 3 * bsz;
#pragma unroll
            for (int kc = 0; kc < HK / 8; ++kc) {
                __nv_bfloat16 hr[8], mr[8], lr[8], hi_[8], mi[8], li[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int qq = kc * 8 + q;
                    const cpx<float> y = conj(tp[nt][qq]) * gsb[hh * HK + qq];
                    accb[nt] = accb[nt] + y;
                    split3(y.x, &hr[q], &mr[q], &lr[q]);
                    split3(y.y, &hi_[q], &mi[q], &li[q]);
                }
                const uint32_t o_re = tc::kmajor_offset(2 * r, hh * HK + kc * 8, KC);
                const uint32_t o_im = tc::kmajor_offset(2 * r + 1, hh * HK + kc * 8, KC);
                *reinterpret_cast<uint4*>(base + o_re) = pack8(hr);
                *reinterpret_cast<uint4*>(base + bsz + o_re) = pack8(mr);
                *reinterpret_cast<uint4*>(base + 2 * bsz + o_re) = pack8(lr);
                *reinterpret_cast<uint4*>(base + o_im) = pack8(hi_);
                *reinterpret_cast<uint4*>(base + bsz + o_im) = pack8(mi);
                *reinterpret_cast<uint4*>(base + 2 * bsz + o_im) = pack8(li);
            }
        }
        if (t == 0)
            for (int q = 0; q < KC; ++q) {
                accg = accg + gsb[q];
                accgg += abs2(gsb[q]);
            }
        if (stage + 1 < nstage) fetch(sb + KC);  // in flight during the MMAs
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            for (int nt = 0; nt < NT; ++nt)
                for (int spl = 0; spl < 3; ++spl)
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint64_t ad = tc::make_desc(tc::smem_u32(As) + ks * 256, 128, 16 * KC);
                        const uint64_t bd = tc::make_desc(
                            tc::smem_u32(Bs + ((size_t)nt * 3 + spl) * bsz) + ks * 256, 128, 16 * KC);
                        tc::mma_bf16(taddr + nt * 256, ad, bd, idesc, (stage | spl | ks) != 0);
                    }
            tc::commit(&mbar[b]);
        }
    }
    // the last commit covers every earlier MMA of this thread
    if (nstage > 0) {
        const int last = nstage - 1;
        ok = tc::mbar_wait(&mbar[last & 1], (last >> 1) & 1, WAIT_LIMIT) && ok;
        tc::fence_after_sync();
    }
    // combine the two walker halves of the a- and b-sums
    red[hh * 128 + r] = acca;
    red[256 + hh * 128 + r] = accb[0];
    __syncthreads();
    cpx<float>* out = (cpx<float>*)partial + (size_t)c * (P + 2 + M);  // float32 rows
    if (hh == 0) {
        if (i < N) out[i] = red[r] + red[128 + r];
        if (blockIdx.y == 0) {
            const int j = r;
            if (j < M) out[N + j] = red[256 + r] + red[384 + r];
        }
    }
    __syncthreads();
    if (NT > 1) {
        red[hh * 128 + r] = accb[1];
        __syncthreads();
        if (hh == 0 && blockIdx.y == 0 && 128 + r < M)
            out[N + 128 + r] = red[r] + red[128 + r];
    }
    if (blockIdx.y == 0 && t == 0) {
        out[P] = accg;
        out[P + 1] = {accgg, 0.f};
    }
    // D rows: warps w and w + 4 read the same TMEM lanes, each half of the columns
    const int lb = warp & 3, half = warp >> 2, row = 32 * lb + lane, ir = i0 + row;
    const int nch16 = NCp / 16;
    for (int nt = 0; nt < NT; ++nt)
        for (int ch = half * (nch16 / 2); ch < (half + 1) * (nch16 / 2) + (half ? nch16 % 2 : 0); ++ch) {
            float d[16];
            tc::tmem_ld16(taddr + ((uint32_t)(32 * lb) << 16) + nt * 256 + ch * 16, d);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = nt * 128 + ch * 8 + q;
                if (ir < N && j < M) out[N + M + (size_t)ir * M + j] = {d[2 * q], d[2 * q + 1]};
            }
        }
    if (!ok && t == 0) set_status(status, CR_ETIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)tmem_cols);
}

// ------------------------------------------------- explicit S (Sec. III)
//
// S_kl = sum_s conj(O_sk) O_sl / B - conj(Obar_k) Obar_l (+ shift on the
// diagonal) through the real Gram matrix G = X^T X of X = [Re O | Im O]
// (column 2k = Re O_k, 2k + 1 = Im O_k):
//   Re S_kl = G[2k][2l] + G[2k+1][2l+1],  Im S_kl = G[2k][2l+1] - G[2k+1][2l].
// Both operands are float32 values split into NPL bf16 terms, the products
// summed in float32 in TMEM over all walkers:
//   NPL = 3 (default): x = hi + mid + lo, six products hi.hi + hi.mid +
//     mid.hi + hi.lo + mid.mid + lo.hi, about float32 accuracy ("bf16x6");
//   NPL = 2 (CR_CTX_S_BF16X3): x = hi + lo + O(2^-17 |x|), three products
//     hi.hi + hi.lo + lo.hi ("bf16x3").  Its error, about 2^-16 relative per
//     product, can push the smallest eigenvalues of S + lambda I below
//     lambda and, at lambda = 1e-3 on large lattices, below zero.
//
// TMEM accumulates in float32 with a per-step error that grows with the
// number of MMAs added into one accumulator (measured: relative ~1e-8 per
// accumulation), so a 128 x 256 tile of G is accumulated over chunks of CH
// walkers in one TMEM half while the other half, holding the previous chunk,
// is added into float32 accumulators in the registers of the drain warps
// (the float64 pipe of this GPU is far too narrow to keep up with the tensor
// cores), which leaves shared memory to a deep operand pipeline.
//
// xt_prep_kernel writes X^T as NPL bf16 planes, each an array of tiles
// [row block of 128 G rows][walker chunk of KC] in the K-major no-swizzle
// core-matrix layout, so one bulk copy moves one tile.
// sgram_tc_kernel: persistent, 288 threads.  Warp 0 (one thread) copies
// operand tiles through NSTG stages (running ahead across tiles) and issues
// the MMAs of chunk c into TMEM columns [256 (c % 2), +256); warps 1-8 wait
// for the chunk, add it to their register tile of S (entries formed from
// adjacent lanes = rows 2k, 2k + 1), release the TMEM half, and at the end
// of a tile write S.
template <int NPL>
struct SGram {
    static constexpr int KC = NPL == 2 ? 32 : 16;    // walkers per operand tile
    static constexpr int TILE = 128 * KC * 2;         // bytes of one 128-row tile
    static constexpr int STAGE = NPL * 3 * TILE;      // A (1 row block) + B (2), NPL planes
    static constexpr int NSTG = NPL == 2 ? 4 : 6;     // pipeline stages
    static constexpr int NPROD = NPL == 2 ? 3 : 6;
    static constexpr int CH = NPL == 2 ? 256 : 128;   // walkers per TMEM accumulation
    static constexpr size_t SMEM = (size_t)NSTG * STAGE + 256;
    // planes (A, B) of product pr: (hi, hi), (hi, mid), (mid, hi), (hi, lo),
    // (mid, mid), (lo, hi); NPL = 2 takes the first three (mid = lo there)
    static CR_HD int pa(int pr) {
        constexpr int v[6] = {0, 0, 1, 0, 1, 2};
        return v[pr];
    }
    static CR_HD int pb(int pr) {
        constexpr int v[6] = {0, 1, 0, 2, 1, 0};
        return v[pr];
    }
};
constexpr int GR_THREADS = 288;

template <int NPL>
__global__ void xt_prep_kernel(const int8_t* __restrict__ spins, const cpx<float>* __restrict__ T,
                               int B, int N, int M, int P, int R2, int nkc_max, int nkc,
                               size_t plane_bytes, unsigned char* __restrict__ Xt) {
    using G = SGram<NPL>;
    constexpr int NG = G::KC / 8;  // groups of 8 walkers per tile
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)R2 * nkc * NG;
    if (idx >= total) return;
    const int r = (int)(idx % 128), grp = (int)((idx / 128) % NG);
    const size_t rest = idx / (128 * NG);
    const int kc = (int)(rest % nkc), rb = (int)(rest / nkc);
    const int row = rb * 128 + r, k = row >> 1, im = row & 1;
    __nv_bfloat16 t0[8], t1[8], t2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int s = kc * G::KC + grp * 8 + q;
        float x = 0.f;
        if (k < P && s < B) {
            cpx<float> o;
            if (k < N) {
                o = {(float)spins[(size_t)s * N + k], 0.f};
            } else if (k < N + M) {
                o = T[(size_t)s * M + (k - N)];
            } else {
                const int i = (k - N - M) / M, j = (k - N - M) % M;
                o = (float)spins[(size_t)s * N + i] * T[(size_t)s * M + j];
            }
            x = im ? o.y : o.x;
        }
        if (NPL == 3) {
            split3(x, &t0[q], &t1[q], &t2[q]);
        } else {
            t0[q] = __float2bfloat16_rn(x);
            t1[q] = __float2bfloat16_rn(x - __bfloat162float(t0[q]));
        }
    }
    const size_t off =
        ((size_t)rb * nkc_max + kc) * G::TILE + tc::kmajor_offset(r, grp * 8, G::KC);
    *reinterpret_cast<uint4*>(Xt + off) = pack8(t0);
    *reinterpret_cast<uint4*>(Xt + plane_bytes + off) = pack8(t1);
    if (NPL == 3) *reinterpret_cast<uint4*>(Xt + 2 * plane_bytes + off) = pack8(t2);
}

// Arguments of sgram_tc_kernel.  A work item is one tile (rt, ct) of G over
// one K segment of kseg walker tiles; items run segment-major (item i:
// segment i / ntiles, tile i % ntiles), so that CTAs running at the same
// time share operand tiles in L2.  tiles[t] = (rt, ct + 65536 op): the
// column operand of op-0 tiles is xb0, of op-1 tiles xb1 (two products with
// one row operand in one launch).  a_exact: the row operand is exact in
// bf16 (spins, ones) and has one plane, so three products (its plane times
// each plane of the column operand) replace the split's six.
struct GramArgs {
    const unsigned char* xa;   // planes of the row operand
    const unsigned char* xb0;  // planes of the column operand of op-0 tiles
    const unsigned char* xb1;  // planes of the column operand of op-1 tiles
    int a_exact;
    size_t plane_bytes;
    int nkc_max;              // walker tiles per row block in the planes
    int kseg, nseg;           // walker tiles per item, K segments per tile
    const int2* tiles;
    int ntiles;
    // explicit S (part == nullptr): S = G / B - conj(Obar) Obar^T + shift I
    int P, B;
    const double* redO;
    double shift;
    double* S;
    // otherwise the raw float32 sums of every item, complex128
    // part[((op * nseg + seg) * Na + n) * Nb + m], n < Na, m < Nb
    double* part;
    int Na, Nb;
    int* status;
};

template <int NPL>
__global__ void __launch_bounds__(GR_THREADS, 1) sgram_tc_kernel(const GramArgs a) {
    using G = SGram<NPL>;
    constexpr int NSTG = G::NSTG, TILE = G::TILE, KPC = G::CH / G::KC;  // tiles per chunk
    const size_t plane_bytes = a.plane_bytes;
    const int nkc_max = a.nkc_max, kseg = a.kseg, ntiles = a.ntiles;
    const int2* __restrict__ tiles = a.tiles;
    int* __restrict__ status = a.status;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* full = (uint64_t*)(sm + NSTG * G::STAGE);
    uint64_t* empty = full + NSTG;      // [NSTG] MMAs reading a stage done
    uint64_t* cdone = full + 2 * NSTG;  // [2] MMAs of a chunk done (per TMEM half)
    uint64_t* drained = cdone + 2;      // [2] TMEM half read by the 256 drain threads
    uint32_t* slot = (uint32_t*)(drained + 2);
    volatile int* abort = (volatile int*)(slot + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        for (int i = 0; i < 2 * NSTG + 2; ++i) tc::mbar_init(&full[i], 1);
        tc::mbar_init(&drained[0], 256);
        tc::mbar_init(&drained[1], 256);
        tc::fence_mbar_init();
        *abort = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, 512u);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;
    const int nchunk = (kseg + KPC - 1) / KPC;
    const int nitems = ntiles * a.nseg;
    const int nmine = nitems > (int)blockIdx.x ? (nitems - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    // a bounded wait that also gives up once the other role has aborted
    auto wait = [&](uint64_t* bar, uint32_t par) {
        for (int i = 0; i < 64; ++i) {
            if (tc::mbar_wait(bar, par, WAIT_LIMIT >> 6)) return true;
            if (*abort) return false;
        }
        *abort = 1;
        return false;
    };
    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------- producer / MMA issuer
            // One flat sequence of stages over all tiles of this CTA, so the
            // copies run NSTG - 1 stages ahead across tile boundaries too.
            const uint32_t idesc = tc::make_idesc_bf16(128, 256);
            const int total = nmine * kseg;
            uint32_t pend = 0, pend_par = 0;
            int last_g = -1;  // last stage whose MMAs were committed
            bool ok = true;
            // copy the operands of stage g; its buffer was last read by the MMAs
            // of stage g - NSTG
            auto load = [&](int g) {
                const uint32_t b = g % NSTG;
                if (g >= NSTG && !wait(&empty[b], ((g - NSTG) / NSTG) & 1)) return false;
                const int item = blockIdx.x + (g / kseg) * gridDim.x;
                const int2 tl = tiles[item % ntiles];
                const int kc = (item / ntiles) * kseg + g % kseg;
                const int rt = tl.x, ct = tl.y & 0xffff;
                const unsigned char* xb = (tl.y >> 16) ? a.xb1 : a.xb0;
                pend |= 1u << b;
                pend_par = (pend_par & ~(1u << b)) | (((uint32_t)(g / NSTG) & 1u) << b);
                unsigned char* st = sm + (size_t)b * G::STAGE;
                const int npa = a.a_exact ? 1 : NPL;  // planes of the row operand
                tc::mbar_expect_tx(&full[b], (uint32_t)((npa + 2 * NPL) * TILE));
                for (int pl = 0; pl < NPL; ++pl) {
                    if (pl < npa)
                        tc::bulk_g2s(st + pl * TILE,
                                     a.xa + (size_t)pl * plane_bytes +
                                         ((size_t)rt * nkc_max + kc) * TILE,
                                     TILE, &full[b]);
                    for (int q = 0; q < 2; ++q)
                        tc::bulk_g2s(st + NPL * TILE + (pl * 2 + q) * TILE,
                                     xb + (size_t)pl * plane_bytes +
                                         ((size_t)(2 * ct + q) * nkc_max + kc) * TILE,
                                     TILE, &full[b]);
                }
                return true;
            };
            for (int g = 0; g < NSTG - 1 && g < total && ok; ++g) ok = load(g);
            for (int g = 0; g < total && ok; ++g) {
                const int kc = g % kseg, b = g % NSTG;
                const int gc = (g / kseg) * nchunk + kc / KPC, first = (kc % KPC) == 0;
                const uint32_t h = gc & 1;
                // the TMEM half of chunk gc was last used by chunk gc - 2
                if (first && gc >= 2 && !wait(&drained[h], ((gc - 2) >> 1) & 1)) {
                    ok = false;
                    break;
                }
                if (!wait(&full[b], (g / NSTG) & 1)) {
                    ok = false;
                    break;
                }
                pend &= ~(1u << b);
                tc::fence_after_sync();
                const unsigned char* st = sm + (size_t)b * G::STAGE;
                const uint32_t a0 = tc::smem_u32(st), b0 = tc::smem_u32(st + NPL * TILE);
                if (a.a_exact) {
#pragma unroll
                    for (int ks = 0; ks < G::KC / 16; ++ks) {
                        const uint64_t ad = tc::make_desc(a0 + ks * 256, 128, 16 * G::KC);
#pragma unroll
                        for (int pl = 0; pl < NPL; ++pl) {
                            const uint64_t bd =
                                tc::make_desc(b0 + pl * 2 * TILE + ks * 256, 128, 16 * G::KC);
                            tc::mma_bf16(taddr + h * 256, ad, bd, idesc, !(first && ks == 0 && pl == 0));
                        }
                    }
                } else {
#pragma unroll
                    for (int ks = 0; ks < G::KC / 16; ++ks) {
#pragma unroll
                        for (int pr = 0; pr < G::NPROD; ++pr) {
                            const uint64_t ad =
                                tc::make_desc(a0 + G::pa(pr) * TILE + ks * 256, 128, 16 * G::KC);
                            const uint64_t bd =
                                tc::make_desc(b0 + G::pb(pr) * 2 * TILE + ks * 256, 128, 16 * G::KC);
                            tc::mma_bf16(taddr + h * 256, ad, bd, idesc,
                                         !(first && ks == 0 && pr == 0));
                        }
                    }
                }
                tc::commit(&empty[b]);
                last_g = g;
                if ((kc + 1) % KPC == 0 || kc + 1 == kseg) tc::commit(&cdone[h]);
                if (g + NSTG - 1 < total && !load(g + NSTG - 1)) ok = false;
            }
            if (!ok) {
                *abort = 1;
                set_status(status, CR_ETIMEOUT);
                // let copies in flight land and issued MMAs finish (bounded)
                for (int b = 0; b < NSTG; ++b)
                    if (pend & (1u << b)) tc::mbar_wait(&full[b], (pend_par >> b) & 1u, WAIT_LIMIT);
                if (last_g >= 0)
                    tc::mbar_wait(&empty[last_g % NSTG], (uint32_t)(last_g / NSTG) & 1u, WAIT_LIMIT);
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ drain (warps 1-8)
        // warp w reads TMEM lanes 32 (w % 4) .. + 31 (G rows) and columns
        // [128 c2, +128) of the chunk's half, c2 = (w - 1) / 4; each lane keeps
        // its 32 entries of S in float32 registers (chunk sums added with
        // round-to-nearest: about sqrt(chunks) 2^-24 on top of each chunk's
        // own error).
        const int lb = warp & 3, c2 = (warp - 1) >> 2, odd = lane & 1;
        const int row = 32 * lb + lane;
        const cpx<double>* redO = (const cpx<double>*)a.redO;
        cpx<double>* S = (cpx<double>*)a.S;
        const int P = a.P;
        const double inv = 1.0 / a.B;
        bool ok = true;
        for (int ti = 0; ti < nmine && ok; ++ti) {
            const int item = blockIdx.x + ti * gridDim.x;
            const int2 tl = tiles[item % ntiles];
            const int rt = tl.x, ct = tl.y & 0xffff;
            float acc[8][4][2];  // [16-column chunk][entry][Re, Im]
#pragma unroll
            for (int ch = 0; ch < 8; ++ch)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[ch][q][0] = acc[ch][q][1] = 0.f;
            for (int ck = 0; ck < nchunk; ++ck) {
                const int gc = ti * nchunk + ck;
                const uint32_t h = gc & 1;
                // warp-uniform outcome: tcgen05.ld below is a warp-wide instruction
                if (!__all_sync(0xffffffffu, wait(&cdone[h], (gc >> 1) & 1))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
#pragma unroll
                for (int ch = 0; ch < 8; ++ch) {
                    float v[16], p[16];
                    tc::tmem_ld16(taddr + ((uint32_t)(32 * lb) << 16) + h * 256 + 128 * c2 + 16 * ch,
                                  v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) p[i] = __shfl_xor_sync(0xffffffffu, v[i], 1);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // even lane: row 2k is its own (v), row 2k+1 the partner's (p); odd: swapped
                        const float e0 = odd ? p[8 + 2 * q] : v[2 * q];
                        const float e1 = odd ? p[9 + 2 * q] : v[2 * q + 1];
                        const float o0 = odd ? v[8 + 2 * q] : p[2 * q];
                        const float o1 = odd ? v[9 + 2 * q] : p[2 * q + 1];
                        acc[ch][q][0] = __fadd_rn(acc[ch][q][0], __fadd_rn(e0, o1));
                        acc[ch][q][1] = __fadd_rn(acc[ch][q][1], __fsub_rn(e1, o0));
                    }
                }
                tc::fence_before_sync();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(
                                 tc::smem_u32(&drained[h]))
                             : "memory");
            }
            if (!ok) break;
            if (a.part) {
                // raw sums of this item: n = row pair, m = column
                const int n = 64 * rt + (row >> 1), Na = a.Na, Nb = a.Nb;
                cpx<double>* out = (cpx<double>*)a.part +
                                   (size_t)((tl.y >> 16) * a.nseg + item / ntiles) * Na * Nb;
                if (n < Na) {
#pragma unroll
                    for (int ch = 0; ch < 8; ++ch)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int m = 128 * ct + 64 * c2 + 8 * ch + 4 * odd + q;
                            if (m < Nb)
                                out[(size_t)n * Nb + m] = {(double)acc[ch][q][0], (double)acc[ch][q][1]};
                        }
                }
                continue;
            }
            // tile done: S = acc / B - conj(Obar_k) Obar_l (+ shift)
            const int k = 64 * rt + (row >> 1);
            if (k < P) {
                const cpx<double> obk = conj(inv * redO[k]);
#pragma unroll
                for (int ch = 0; ch < 8; ++ch)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int l = 128 * ct + 64 * c2 + 8 * ch + 4 * odd + q;
                        if (l < P) {
                            const cpx<double> g = {(double)acc[ch][q][0], (double)acc[ch][q][1]};
                            cpx<double> val = inv * g - obk * (inv * redO[l]);
                            if (k == l) val.x += a.shift;
                            S[(size_t)k * P + l] = val;
                        }
                    }
            }
        }
        if (!ok && t == 32) set_status(status, CR_ETIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, 512u);
}

// S[k][l] = conj(S[l][k]) for k < l (32 x 32 tiles through shared memory).
__global__ void smirror_kernel(double* __restrict__ S_, int P) {
    __shared__ cpx<double> tl[32][33];
    const int bx = blockIdx.x, by = blockIdx.y;  // tile column, tile row
    if (bx < by) return;                         // tiles on or above the diagonal only
    cpx<double>* S = (cpx<double>*)S_;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int j = ty; j < 32; j += 8) {
        const int r = bx * 32 + j, c = by * 32 + tx;  // source: lower block (row bx, col by)
        if (r < P && c < P) tl[j][tx] = S[(size_t)r * P + c];
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const int r = by * 32 + j, c = bx * 32 + tx;  // destination (row by, col bx)
        if (r < P && c < P && r < c) S[(size_t)r * P + c] = conj(tl[tx][j]);
    }
}

// ---------------------------------------------- Krylov Gram (Sec. IV)
//
// G = B^dag B / B_s and H = B^dag HB / B_s of cheb_gram on the tensor cores:
// the complex columns B_n (and HB_n) become rows 2n (real part) and 2n + 1
// (imaginary part) of a real matrix X (Y), split into three bf16 planes as
// for the explicit S, and sgram_tc_kernel forms X^T X and X^T Y over K
// segments of the samples.  gram_reduce_kernel adds the segments in float64
// in a fixed order, scales by 1/B_s, and writes G (Hermitian by construction:
// upper triangle mirrored, real diagonal) and (H + H^dag)/2.

// Planes of X from the columns Bm[n * ld + s] (complex64): row 2n + im,
// walkers s; rows past 2 Nm and walkers past B are zero.
template <int NPL>
__global__ void gram_prep_kernel(const cpx<float>* __restrict__ Bm, int Nm, int B, int ld, int nrb,
                                 int nkc, size_t plane_bytes, unsigned char* __restrict__ X) {
    using G = SGram<NPL>;
    constexpr int NG = G::KC / 8;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nrb * nkc * NG * 128) return;
    const int r = (int)(idx % 128), grp = (int)((idx / 128) % NG);
    const size_t rest = idx / (128 * NG);
    const int kc = (int)(rest % nkc), rb = (int)(rest / nkc);
    const int row = rb * 128 + r, n = row >> 1, im = row & 1;
    __nv_bfloat16 t0[8], t1[8], t2[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int s = kc * G::KC + grp * 8 + q;
        float x = 0.f;
        if (n < Nm && s < B) {
            const cpx<float> v = Bm[(size_t)n * ld + s];
            x = im ? v.y : v.x;
        }
        if (NPL == 3) {
            split3(x, &t0[q], &t1[q], &t2[q]);
        } else {
            t0[q] = __float2bfloat16_rn(x);
            t1[q] = __float2bfloat16_rn(x - __bfloat162float(t0[q]));
        }
    }
    const size_t off = ((size_t)rb * nkc + kc) * G::TILE + tc::kmajor_offset(r, grp * 8, G::KC);
    *reinterpret_cast<uint4*>(X + off) = pack8(t0);
    *reinterpret_cast<uint4*>(X + plane_bytes + off) = pack8(t1);
    if (NPL == 3) *reinterpret_cast<uint4*>(X + 2 * plane_bytes + off) = pack8(t2);
}

__global__ void gram_reduce_kernel(const double* __restrict__ part_, int nseg, int Nm, int B,
                                   double* __restrict__ G_, double* __restrict__ H_) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Nm * Nm) return;
    const int n = idx / Nm, m = idx % Nm;
    if (m < n) return;
    const cpx<double>* part = (const cpx<double>*)part_;
    const size_t NN = (size_t)Nm * Nm;
    const double inv = 1.0 / B;
    cpx<double> g = {0.0, 0.0};
    for (int sg = 0; sg < nseg; ++sg) g = g + part[sg * NN + (size_t)n * Nm + m];
    g = inv * g;
    if (n == m) g.y = 0.0;
    cpx<double>* Gc = (cpx<double>*)G_;
    Gc[(size_t)n * Nm + m] = g;
    Gc[(size_t)m * Nm + n] = conj(g);
    if (H_) {
        cpx<double> h1 = {0.0, 0.0}, h2 = {0.0, 0.0};
        for (int sg = 0; sg < nseg; ++sg) {
            h1 = h1 + part[(nseg + sg) * NN + (size_t)n * Nm + m];
            h2 = h2 + part[(nseg + sg) * NN + (size_t)m * Nm + n];
        }
        const cpx<double> v = (0.5 * inv) * (h1 + conj(h2));
        cpx<double>* Hc = (cpx<double>*)H_;
        Hc[(size_t)n * Nm + m] = v;
        Hc[(size_t)m * Nm + n] = conj(v);
    }
}

// ------------------------------------------------------------ launchers

static int tc_geometry(int M, int* NCp, int* NT) {
    *NT = (M + 127) / 128;
    const int w = 2 * (M < 128 ? M : 128);
    *NCp = ((w + 15) / 16) * 16;
    return *NT == 1 ? 256 : 512;  // TMEM columns (power of two)
}

size_t ov_tc_smem(const cr_ctx* c) {
    int NCp, NT;
    tc_geometry(c->M, &NCp, &NT);
    const int Kp = ((c->N + 15) / 16) * 16;
    return (size_t)NT * 3 * NCp * Kp * 2 + (size_t)128 * Kp * 2 +
           (size_t)2 * 128 * (TJC + 1) * 8 + (size_t)(c->M + c->N + 256) * 8 + 64;
}

size_t oreduce_tc_smem(const cr_ctx* c) {
    int NCp, NT;
    tc_geometry(c->M, &NCp, &NT);
    return 2 * ((size_t)NT * 3 * NCp * 32 * 2 + 128 * 32 * 2) + 2 * 32 * 8 + 4 * 128 * 8 + 64;
}

// Whether the tensor-core kernels cover this context (M <= 256 and the
// operands fit in shared memory); otherwise the float32 kernels run.
// Shared-memory bound of the tensor-core kernels.  The kernels' opt-in limit
// is set to this bound, not to one context's need: the attribute belongs to
// the function, so a context created later with a smaller need must not
// lower it under an earlier context's launches.
constexpr int TC_SMEM_LIMIT = 200 * 1024;

bool tc_supported(const cr_ctx* c) {
    return c->prec == CR_MIXED && c->M <= 256 && ov_tc_smem(c) <= TC_SMEM_LIMIT &&
           oreduce_tc_smem(c) <= TC_SMEM_LIMIT;
}

cr_status launch_ov_tc(cr_ctx* c, const void* v, const int8_t* spins, int B, const void* T,
                       void* u, const double* skip) {
    int NCp, NT;
    const int cols = tc_geometry(c->M, &NCp, &NT);
    const int Kp = ((c->N + 15) / 16) * 16;
    const size_t sm = ov_tc_smem(c);
    const int ntiles = (B + 127) / 128;
    const int grid = ntiles < c->n_sm ? ntiles : c->n_sm;
    CR_LAUNCH(c, CR_KERNEL_OV,
              ov_tc_kernel<<<grid, OV_THREADS, sm, c->stream>>>(
                  (const cpx<float>*)v, spins, (const cpx<float>*)T, B, c->N, c->M, Kp, NCp, NT,
                  cols, (cpx<float>*)u, skip, c->d_status));
    return cr_check_launch(c, "ov_tc_kernel");
}

// Returns the number of chunk rows written (every chunk non-empty).
cr_status launch_oreduce_tc(cr_ctx* c, const int8_t* spins, const void* T, const void* g, int B,
                            const double* skip, int* nch_out) {
    int NCp, NT;
    const int cols = tc_geometry(c->M, &NCp, &NT);
    int nch0 = (B + 31) / 32;
    if (nch0 > c->n_chunks) nch0 = c->n_chunks;
    const int chunk = (B + nch0 - 1) / nch0;
    const int nch = (B + chunk - 1) / chunk;
    const size_t sm = oreduce_tc_smem(c);
    CR_LAUNCH(c, CR_KERNEL_REDUCE,
              oreduce_tc_kernel<<<dim3(nch, (c->N + 127) / 128), RED_THREADS, sm, c->stream>>>(
                  spins, (const cpx<float>*)T, (const cpx<float>*)g, B, c->N, c->M, c->P, chunk,
                  NCp, NT, cols, c->partial, skip, c->d_status));
    *nch_out = nch;
    return cr_check_launch(c, "oreduce_tc_kernel");
}

static int sgram_npl(const cr_ctx* c) { return (c->flags & CR_CTX_S_BF16X3) ? 2 : 3; }

template <int NPL> size_t sgram_smem_t() { return SGram<NPL>::SMEM; }

// Operand planes of the explicit-S Gram kernel: rows of G padded to a
// multiple of 512, walkers to a multiple of the tile's walker count.
void sgram_geometry(const cr_ctx* c, int* R2, int* nkc_max, size_t* plane_bytes, int* npl) {
    *npl = sgram_npl(c);
    const int kc = *npl == 2 ? SGram<2>::KC : SGram<3>::KC;
    *R2 = ((2 * c->P + 511) / 512) * 512;
    *nkc_max = (c->max_walkers + kc - 1) / kc;
    *plane_bytes = (size_t)(*R2 / 128) * (size_t)(*nkc_max) * (size_t)(128 * kc * 2);
}

// Lower-triangle blocks of G (128-row block rt, 256-column block ct with
// 256 ct <= 128 rt + 127), column-block major so that concurrently running
// CTAs share the column operand in L2.
std::vector<int2> sgram_tiles(int P) {
    const int R2 = ((2 * P + 511) / 512) * 512;
    std::vector<int2> v;
    for (int ct = 0; ct < R2 / 256; ++ct)
        for (int rt = 0; rt * 128 < 2 * P; ++rt)
            if (256 * ct <= 128 * rt + 127) v.push_back(make_int2(rt, ct));
    return v;
}

void launch_smirror(cr_ctx* c);

template <int NPL>
static cr_status sbuild_tc_t(cr_ctx* c, const int8_t* spins, const void* T, int B,
                             const double* redO, double shift) {
    int R2, nkc_max, npl;
    size_t pb;
    sgram_geometry(c, &R2, &nkc_max, &pb, &npl);
    constexpr int KC = SGram<NPL>::KC;
    const int nkc = (B + KC - 1) / KC;
    const size_t n = (size_t)R2 * nkc * (KC / 8);
    CR_LAUNCH(c, CR_K_OTHER,
              xt_prep_kernel<NPL><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                  spins, (const cpx<float>*)T, B, c->N, c->M, c->P, R2, nkc_max, nkc, pb, c->Xt));
    const int grid = c->n_gtiles < c->n_sm ? c->n_gtiles : c->n_sm;
    GramArgs a{};
    a.xa = a.xb0 = a.xb1 = c->Xt;
    a.plane_bytes = pb;
    a.nkc_max = nkc_max;
    a.kseg = nkc;
    a.nseg = 1;
    a.tiles = c->gtiles;
    a.ntiles = c->n_gtiles;
    a.P = c->P;
    a.B = B;
    a.redO = redO;
    a.shift = shift;
    a.S = c->S;
    a.status = c->d_status;
    CR_LAUNCH(c, CR_KERNEL_SBUILD,
              sgram_tc_kernel<NPL><<<grid, GR_THREADS, sgram_smem_t<NPL>(), c->stream>>>(a));
    launch_smirror(c);
    return cr_check_launch(c, "explicit S (tensor cores)");
}

cr_status launch_sbuild_tc(cr_ctx* c, const int8_t* spins, const void* T, int B,
                           const double* redO, double shift) {
    return sgram_npl(c) == 2 ? sbuild_tc_t<2>(c, spins, T, B, redO, shift)
                             : sbuild_tc_t<3>(c, spins, T, B, redO, shift);
}

void launch_smirror(cr_ctx* c) {
    const int nt = (c->P + 31) / 32;
    CR_LAUNCH(c, CR_K_OTHER, smirror_kernel<<<dim3(nt, nt), dim3(32, 8), 0, c->stream>>>(c->S, c->P));
}

// Geometry of the Krylov Gram on the tensor cores (three-plane split): rows
// of X padded to a multiple of 256, the items' K segments of equal length
// (walker tiles past B are zero), G tiles on and above the diagonal, all H
// tiles.
struct GramGeo {
    int nrb, nseg, kseg, nkc;
    size_t plane_bytes, x_bytes, part_bytes;
    std::vector<int2> tiles;
};

static GramGeo gram_geometry(const cr_ctx* c, int Nm, int B, bool withH) {
    using G = SGram<3>;
    constexpr int KPC = G::CH / G::KC;
    GramGeo g;
    const int R2 = ((2 * Nm + 255) / 256) * 256;
    g.nrb = R2 / 128;
    const int nrt = (2 * Nm + 127) / 128;
    for (int op = 0; op < (withH ? 2 : 1); ++op)
        for (int ct = 0; ct < R2 / 256; ++ct)
            for (int rt = 0; rt < nrt; ++rt)
                if (op == 1 || 64 * rt <= 128 * ct + 127) g.tiles.push_back(make_int2(rt, ct + 65536 * op));
    const int nt = (int)g.tiles.size();
    const int nch = (B + G::CH - 1) / G::CH;  // 128-walker chunks
    int nseg = c->n_sm / nt;
    if (nseg > nch / 4) nseg = nch / 4;      // at least 4 chunks per segment
    if (nseg < 1) nseg = 1;
    const int cps = (nch + nseg - 1) / nseg;  // chunks per segment
    g.nseg = (nch + cps - 1) / cps;
    g.kseg = cps * KPC;
    g.nkc = g.nseg * g.kseg;
    g.plane_bytes = (size_t)g.nrb * g.nkc * G::TILE;
    g.x_bytes = (withH ? 2 : 1) * 3 * g.plane_bytes;
    g.part_bytes = (size_t)(withH ? 2 : 1) * g.nseg * Nm * Nm * 16;
    return g;
}

cr_status launch_gram_tc(cr_ctx* c, const void* Bm, const void* HBm, int Nm, int B, int ld,
                         double* G, double* H) {
    GramGeo g = gram_geometry(c, Nm, B, HBm != nullptr);
    cr_status st = cr_grow(c, (void**)&c->gram_x, &c->gram_x_cap, g.x_bytes, "cheb_gram");
    if (st == CR_OK) st = cr_grow(c, (void**)&c->gram_part, &c->gram_part_cap, g.part_bytes, "cheb_gram");
    const size_t tcap = c->gram_tiles_cap;
    if (st == CR_OK)
        st = cr_grow(c, (void**)&c->gram_tiles, &c->gram_tiles_cap, g.tiles.size() * sizeof(int2),
                     "cheb_gram");
    if (c->gram_tiles_cap != tcap) c->gram_key = 0;
    if (st != CR_OK) return st;
    const int key = 2 * Nm + (HBm ? 1 : 0);
    if (c->gram_key != key) {
        // the tile list changes with Nm only (pageable source: staged before return)
        if (cudaMemcpyAsync(c->gram_tiles, g.tiles.data(), g.tiles.size() * sizeof(int2),
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
            return cr_fail(c, CR_ECUDA, "cheb_gram: tile list copy");
        c->gram_key = key;
    }
    constexpr int NG = SGram<3>::KC / 8;
    const size_t n = (size_t)g.nrb * g.nkc * NG * 128;
    const unsigned nb = (unsigned)((n + 255) / 256);
    unsigned char* X = c->gram_x;
    unsigned char* Y = HBm ? X + 3 * g.plane_bytes : X;
    CR_LAUNCH(c, CR_K_OTHER, gram_prep_kernel<3><<<nb, 256, 0, c->stream>>>(
                                 (const cpx<float>*)Bm, Nm, B, ld, g.nrb, g.nkc, g.plane_bytes, X));
    if (HBm)
        CR_LAUNCH(c, CR_K_OTHER, gram_prep_kernel<3><<<nb, 256, 0, c->stream>>>(
                                     (const cpx<float>*)HBm, Nm, B, ld, g.nrb, g.nkc, g.plane_bytes, Y));
    GramArgs a{};
    a.xa = a.xb0 = X;
    a.xb1 = Y;
    a.plane_bytes = g.plane_bytes;
    a.nkc_max = g.nkc;
    a.kseg = g.kseg;
    a.nseg = g.nseg;
    a.tiles = c->gram_tiles;
    a.ntiles = (int)g.tiles.size();
    a.B = B;
    a.part = c->gram_part;
    a.Na = a.Nb = Nm;
    a.status = c->d_status;
    const int items = a.ntiles * a.nseg;
    const int grid = items < c->n_sm ? items : c->n_sm;
    CR_LAUNCH(c, CR_KERNEL_GRAM,
              sgram_tc_kernel<3><<<grid, GR_THREADS, sgram_smem_t<3>(), c->stream>>>(a));
    CR_LAUNCH(c, CR_K_OTHER, gram_reduce_kernel<<<(Nm * Nm + 255) / 256, 256, 0, c->stream>>>(
                                 c->gram_part, g.nseg, Nm, B, G, H));
    return cr_check_launch(c, "cheb_gram (tensor cores)");
}

// ------------------------------------ estimator sums on the tensor cores
//
// The two walker sums of a natural-gradient step (Sec. III),
//   redR = [sum sigma_i g | sum conj(T_j) g | sum sigma_i conj(T_j) g | sum g | sum |g|^2]
//   redO = [sum sigma_i   | sum T_j         | sum sigma_i T_j         | B     | B      ]
// (g = R; the layout of oreduce's rows), as one launch of sgram_tc_kernel:
// row operand A = [sigma_0 .. sigma_{N-1}, 1] (exact in bf16: one plane),
// column operands Y0 = [conj(T_j) g, g, |g|^2] (op 0) and Y1 = [T_j, 1]
// (op 1), split into three bf16 planes; out = sum_s A_k(s) Y_l(s) over K
// segments, added in float64 by ored_reduce_kernel.  The sums of |T_j|^2
// (the Jacobi diagonal) are not formed here.
struct OredGeo {
    int R2, nrb, nseg, nkc_cap, Na, Nb;
    size_t plane_bytes, x_bytes, part_bytes;
    std::vector<int2> tiles;
};

static OredGeo ored_geometry(const cr_ctx* c) {
    using G = SGram<3>;
    constexpr int KPC = G::CH / G::KC;
    OredGeo g;
    g.Na = c->N + 1;
    g.Nb = c->M + 2;
    const int ra = 2 * g.Na, rb0 = 2 * (c->M + 2), rb1 = 2 * (c->M + 1);
    const int rmax = ra > rb0 ? ra : rb0;
    g.R2 = ((rmax + 255) / 256) * 256;
    g.nrb = g.R2 / 128;
    const int nrt = (ra + 127) / 128;
    for (int op = 0; op < 2; ++op) {
        const int nct = ((op ? rb1 : rb0) + 255) / 256;
        for (int ct = 0; ct < nct; ++ct)
            for (int rt = 0; rt < nrt; ++rt) g.tiles.push_back(make_int2(rt, ct + 65536 * op));
    }
    const int nt = (int)g.tiles.size();
    g.nseg = c->n_sm / nt > 1 ? c->n_sm / nt : 1;
    const int nch = (c->max_walkers + G::CH - 1) / G::CH;
    g.nkc_cap = g.nseg * ((nch + g.nseg - 1) / g.nseg) * KPC;
    g.plane_bytes = (size_t)g.nrb * g.nkc_cap * G::TILE;
    g.x_bytes = 7 * g.plane_bytes;  // A: one plane; Y0, Y1: three each
    g.part_bytes = (size_t)2 * g.nseg * g.Na * g.Nb * 16;
    return g;
}

void ored_sizes(const cr_ctx* c, size_t* x_bytes, size_t* part_bytes, std::vector<int2>* tiles) {
    OredGeo g = ored_geometry(c);
    *x_bytes = g.x_bytes;
    *part_bytes = g.part_bytes;
    *tiles = g.tiles;
}

// Planes of A (plane 0 only) and of Y0, Y1 for walker tiles kc < nkc (zero
// past B): one thread per (row, 8 walkers); T is read once for both Y.
__global__ void ored_prep_kernel(const int8_t* __restrict__ spins, const cpx<float>* __restrict__ T,
                                 const cpx<float>* __restrict__ g, int B, int N, int M, int nrb,
                                 int nkc, int nkc_cap, size_t plane_bytes,
                                 unsigned char* __restrict__ X) {
    using G = SGram<3>;
    constexpr int NG = G::KC / 8;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)nrb * nkc * NG * 128) return;
    const int r = (int)(idx % 128), grp = (int)((idx / 128) % NG);
    const size_t rest = idx / (128 * NG);
    const int kc = (int)(rest % nkc), rb = (int)(rest / nkc);
    const int row = rb * 128 + r, k = row >> 1, im = row & 1;
    __nv_bfloat16 a[8], y0[3][8], y1[3][8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int s = kc * G::KC + grp * 8 + q;
        float xa = 0.f, x0 = 0.f, x1 = 0.f;
        if (s < B) {
            if (!im) xa = k < N ? (float)spins[(size_t)s * N + k] : (k == N ? 1.f : 0.f);
            const cpx<float> gs = g[s];
            cpx<float> v0 = {0.f, 0.f}, v1 = {0.f, 0.f};
            if (k < M) {
                const cpx<float> t = T[(size_t)s * M + k];
                v0 = conj(t) * gs;
                v1 = t;
            } else if (k == M) {
                v0 = gs;
                v1 = {1.f, 0.f};
            } else if (k == M + 1) {
                v0 = {abs2(gs), 0.f};
            }
            x0 = im ? v0.y : v0.x;
            x1 = im ? v1.y : v1.x;
        }
        a[q] = __float2bfloat16_rn(xa);  // exact: +-1, 1 or 0
        split3(x0, &y0[0][q], &y0[1][q], &y0[2][q]);
        split3(x1, &y1[0][q], &y1[1][q], &y1[2][q]);
    }
    const size_t off = ((size_t)rb * nkc_cap + kc) * G::TILE + tc::kmajor_offset(r, grp * 8, G::KC);
    *reinterpret_cast<uint4*>(X + off) = pack8(a);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
        *reinterpret_cast<uint4*>(X + (1 + pl) * plane_bytes + off) = pack8(y0[pl]);
        *reinterpret_cast<uint4*>(X + (4 + pl) * plane_bytes + off) = pack8(y1[pl]);
    }
}

__global__ void ored_reduce_kernel(const double* __restrict__ part_, int nseg, int N, int M, int P,
                                   int Na, int Nb, double* __restrict__ redR_,
                                   double* __restrict__ redO_) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P + 2 + M) return;
    cpx<double>* redR = (cpx<double>*)redR_;
    cpx<double>* redO = (cpx<double>*)redO_;
    if (k >= P + 2) {
        redO[k] = {0.0, 0.0};  // sums of |T_j|^2: not formed on this path
        return;
    }
    int n, m;  // (row of A, column of Y)
    if (k < N) { n = k; m = M; }
    else if (k < N + M) { n = N; m = k - N; }
    else if (k < P) { n = (k - N - M) / M; m = (k - N - M) % M; }
    else { n = N; m = M + (k - P); }
    const cpx<double>* part = (const cpx<double>*)part_;
    const size_t NN = (size_t)Na * Nb, e = (size_t)n * Nb + m;
    cpx<double> r = {0.0, 0.0}, o = {0.0, 0.0};
    for (int sg = 0; sg < nseg; ++sg) {
        r = r + part[sg * NN + e];
        if (k <= P) o = o + part[(nseg + sg) * NN + e];
    }
    if (k == P + 1) {
        // sum |1|^2 = sum 1, the B of entry P
        for (int sg = 0; sg < nseg; ++sg) o = o + part[(nseg + sg) * NN + (size_t)N * Nb + M];
        r.y = 0.0;
    }
    redR[k] = r;
    redO[k] = o;
}

cr_status launch_oreduce_tc(cr_ctx* c, const int8_t* spins, const void* T, const void* g, int B,
                            double* redR, double* redO) {
    using G = SGram<3>;
    constexpr int KPC = G::CH / G::KC, NG = G::KC / 8;
    OredGeo geo = ored_geometry(c);
    const int nch = (B + G::CH - 1) / G::CH;
    const int cps = (nch + geo.nseg - 1) / geo.nseg;
    const int nseg = (nch + cps - 1) / cps, kseg = cps * KPC, nkc = nseg * kseg;
    const size_t n = (size_t)geo.nrb * nkc * NG * 128;
    CR_LAUNCH(c, CR_K_OTHER, ored_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                                 spins, (const cpx<float>*)T, (const cpx<float>*)g, B, c->N, c->M,
                                 geo.nrb, nkc, geo.nkc_cap, geo.plane_bytes, c->ored_x));
    GramArgs a{};
    a.xa = c->ored_x;
    a.xb0 = c->ored_x + geo.plane_bytes;
    a.xb1 = c->ored_x + 4 * geo.plane_bytes;
    a.a_exact = 1;
    a.plane_bytes = geo.plane_bytes;
    a.nkc_max = geo.nkc_cap;
    a.kseg = kseg;
    a.nseg = nseg;
    a.tiles = c->ored_tiles;
    a.ntiles = (int)geo.tiles.size();
    a.B = B;
    a.part = c->ored_part;
    a.Na = geo.Na;
    a.Nb = geo.Nb;
    a.status = c->d_status;
    const int items = a.ntiles * nseg;
    const int grid = items < c->n_sm ? items : c->n_sm;
    CR_LAUNCH(c, CR_KERNEL_REDUCE,
              sgram_tc_kernel<3><<<grid, GR_THREADS, sgram_smem_t<3>(), c->stream>>>(a));
    const int len = c->P + 2 + c->M;
    CR_LAUNCH(c, CR_K_OTHER, ored_reduce_kernel<<<(len + 255) / 256, 256, 0, c->stream>>>(
                                 c->ored_part, nseg, c->N, c->M, c->P, geo.Na, geo.Nb, redR, redO));
    return cr_check_launch(c, "estimator sums (tensor cores)");
}

// Opt the tensor-core kernels into the shared memory they need; called once
// per context (not from a hot call, so that hot calls stay capturable).
cr_status tc_prepare(cr_ctx* c) {
    if (c->prec == CR_MIXED) {
        // explicit S (either split) and the Krylov Gram (three planes)
        cudaError_t e = cudaFuncSetAttribute(sgram_tc_kernel<2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sgram_smem_t<2>());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sgram_tc_kernel<3>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sgram_smem_t<3>());
        if (e != cudaSuccess) return cr_fail(c, CR_ECUDA, "tc_prepare: %s", cudaGetErrorString(e));
    }
    if (!tc_supported(c)) return CR_OK;
    cudaError_t e = cudaFuncSetAttribute(ov_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TC_SMEM_LIMIT);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(oreduce_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TC_SMEM_LIMIT);
    return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "tc_prepare: %s", cudaGetErrorString(e));
}
