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
#include <cuda_bf16.h>

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
// Shared memory: Bs [NT][3][NCp x Kp] (V_W split, column n = 2 j + re/im,
// K = sites), As [128 x Kp] (the spins of one 128-walker tile), vb [M],
// va [N], one mbarrier and the TMEM address slot.  A CTA loops over walker
// tiles; D = sigma V for a tile occupies TMEM columns [256 nt, 256 nt + NCp).
__global__ void __launch_bounds__(128, 1) ov_tc_kernel(
    const cpx<float>* __restrict__ v, const int8_t* __restrict__ spins,
    const cpx<float>* __restrict__ T, int B, int N, int M, int Kp, int NCp, int NT,
    int tmem_cols, cpx<float>* __restrict__ u, const double* __restrict__ skip,
    int* __restrict__ status) {
    if (skip && *skip != 0.0) return;
    extern __shared__ __align__(1024) unsigned char sm[];
    const size_t bsz = (size_t)NCp * Kp * 2;          // one split of one n-tile
    unsigned char* Bs = sm;
    unsigned char* As = sm + (size_t)NT * 3 * bsz;
    cpx<float>* vb = (cpx<float>*)(As + (size_t)128 * Kp * 2);
    cpx<float>* va = vb + M;
    uint64_t* mbar = (uint64_t*)(((uintptr_t)(va + N) + 15) & ~(uintptr_t)15);
    uint32_t* slot = (uint32_t*)(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5;
    if (t == 0) {
        tc::mbar_init(mbar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, (uint32_t)tmem_cols);
        tc::tmem_relinquish();
    }
    // V_W in three bf16 terms, K-major (sites contiguous per column)
    const int kc_n = Kp / 8;
    for (int e = t; e < NT * NCp * kc_n; e += 128) {
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
    for (int j = t; j < M; j += 128) vb[j] = v[N + j];
    for (int i = t; i < N; i += 128) va[i] = v[i];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = *slot;
    const uint32_t idesc = tc::make_idesc_bf16(128, NCp);
    const int ntiles = (B + 127) / 128;
    bool ok = true;
    int it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
        const int w = tile * 128 + t;
        cpx<float> ua = {0.f, 0.f};
        for (int kc = 0; kc < kc_n; ++kc) {
            __nv_bfloat16 s8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = kc * 8 + q;
                const int sv = (w < B && k < N) ? spins[(size_t)w * N + k] : 0;
                s8[q] = __float2bfloat16_rn((float)sv);
                if (sv) ua = ua + (float)sv * va[k];
            }
            *reinterpret_cast<uint4*>(As + tc::kmajor_offset(t, kc * 8, Kp)) = pack8(s8);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();  // As written; the previous tile's TMEM reads are done
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
        ok = tc::mbar_wait(mbar, it & 1, WAIT_LIMIT) && ok;
        tc::fence_after_sync();
        cpx<float> acc = ua;
        for (int nt = 0; nt < NT; ++nt)
            for (int ch = 0; ch < NCp / 16; ++ch) {
                float d[16];
                tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + nt * 256 + ch * 16, d);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int j = nt * 128 + ch * 8 + q;
                    if (j < M && w < B) {
                        cpx<float> x = {d[2 * q] + vb[j].x, d[2 * q + 1] + vb[j].y};
                        acc = acc + T[(size_t)w * M + j] * x;
                    }
                }
            }
        if (w < B) u[w] = acc;
    }
    if (!ok && t == 0) set_status(status, CR_ETIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)tmem_cols);
}

// ------------------------------------------------------- O^dag g reduction
//
// One CTA per (walker chunk, tile of 128 sites).  Per stage of 32 walkers:
// As [128 x 32] = sigma^T (sites x walkers), Bs [NT][3][NCp x 32] = the bf16
// terms of Y^T, Y_sj = conj(T_sj) g_s.  D accumulates over the chunk in TMEM.
__global__ void __launch_bounds__(128, 1) oreduce_tc_kernel(
    const int8_t* __restrict__ spins, const cpx<float>* __restrict__ T,
    const cpx<float>* __restrict__ g, int B, int N, int M, int P, int chunk, int NCp, int NT,
    int tmem_cols, double* __restrict__ partial, const double* __restrict__ skip,
    int* __restrict__ status) {
    if (skip && *skip != 0.0) return;
    constexpr int KC = 32;
    extern __shared__ __align__(1024) unsigned char sm[];
    const size_t bsz = (size_t)NCp * KC * 2;
    unsigned char* Bs = sm;
    unsigned char* As = sm + (size_t)NT * 3 * bsz;
    cpx<float>* gs = (cpx<float>*)(As + 128 * KC * 2);
    uint64_t* mbar = (uint64_t*)(gs + KC);
    uint32_t* slot = (uint32_t*)(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5;
    const int c = blockIdx.x, i0 = blockIdx.y * 128;
    const int s0 = c * chunk, s1 = min(B, s0 + chunk);
    if (t == 0) {
        tc::mbar_init(mbar, 1);
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
    int stage = 0;
    for (int sb = s0; sb < s1; sb += KC, ++stage) {
        if (t < KC) {
            const int s = sb + t;
            gs[t] = s < s1 ? g[s] : cpx<float>{0.f, 0.f};
        }
        __syncthreads();
        // sigma^T: row t = site i0 + t, 32 walkers
        const int i = i0 + t;
        for (int kc = 0; kc < KC / 8; ++kc) {
            __nv_bfloat16 s8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int s = sb + kc * 8 + q;
                const int sv = (s < s1 && i < N) ? spins[(size_t)s * N + i] : 0;
                s8[q] = __float2bfloat16_rn((float)sv);
                if (sv) acca = acca + (float)sv * gs[kc * 8 + q];
            }
            *reinterpret_cast<uint4*>(As + tc::kmajor_offset(t, kc * 8, KC)) = pack8(s8);
        }
        // Y^T: complex column j = 128 nt + t (real columns 2t, 2t + 1 of n-tile nt)
        for (int nt = 0; nt < NT; ++nt) {
            const int j = nt * 128 + t;
            if (2 * t >= NCp) break;  // columns past NCp do not exist in this tile
            for (int kc = 0; kc < KC / 8; ++kc) {
                __nv_bfloat16 hr[8], mr[8], lr[8], hi_[8], mi[8], li[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int s = sb + kc * 8 + q;
                    cpx<float> y = {0.f, 0.f};
                    if (s < s1 && j < M) y = conj(T[(size_t)s * M + j]) * gs[kc * 8 + q];
                    accb[nt] = accb[nt] + y;
                    split3(y.x, &hr[q], &mr[q], &lr[q]);
                    split3(y.y, &hi_[q], &mi[q], &li[q]);
                }
                unsigned char* base = Bs + (size_t)nt * 3 * bsz;
                const uint32_t o_re = tc::kmajor_offset(2 * t, kc * 8, KC);
                const uint32_t o_im = tc::kmajor_offset(2 * t + 1, kc * 8, KC);
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
                accg = accg + gs[q];
                accgg += abs2(gs[q]);
            }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0) {
            for (int nt = 0; nt < NT; ++nt)
                for (int sp = 0; sp < 3; ++sp)
                    for (int ks = 0; ks < KC / 16; ++ks) {
                        const uint64_t ad = tc::make_desc(tc::smem_u32(As) + ks * 256, 128, 16 * KC);
                        const uint64_t bd = tc::make_desc(
                            tc::smem_u32(Bs + ((size_t)nt * 3 + sp) * bsz) + ks * 256, 128, 16 * KC);
                        tc::mma_bf16(taddr + nt * 256, ad, bd, idesc, (stage | sp | ks) != 0);
                    }
            tc::commit(mbar);
        }
        // the operands are rewritten next stage: wait for these MMAs
        ok = tc::mbar_wait(mbar, stage & 1, WAIT_LIMIT) && ok;
        tc::fence_after_sync();
    }
    cpx<double>* out = (cpx<double>*)partial + (size_t)c * (P + 2 + M);
    // D row t = site i0 + t
    const int i = i0 + t;
    for (int nt = 0; nt < NT; ++nt)
        for (int ch = 0; ch < NCp / 16; ++ch) {
            float d[16];
            tc::tmem_ld16(taddr + ((uint32_t)(32 * warp) << 16) + nt * 256 + ch * 16, d);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int j = nt * 128 + ch * 8 + q;
                if (i < N && j < M)
                    out[N + M + (size_t)i * M + j] = {(double)d[2 * q], (double)d[2 * q + 1]};
            }
        }
    if (i < N) out[i] = ccast<double>(acca);
    if (blockIdx.y == 0) {
        for (int nt = 0; nt < NT; ++nt) {
            const int j = nt * 128 + t;
            if (j < M) out[N + j] = ccast<double>(accb[nt]);
        }
        if (t == 0) {
            out[P] = ccast<double>(accg);
            out[P + 1] = {(double)accgg, 0.0};
        }
    }
    if (!ok && t == 0) set_status(status, CR_ETIMEOUT);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(taddr, (uint32_t)tmem_cols);
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
    return (size_t)NT * 3 * NCp * Kp * 2 + (size_t)128 * Kp * 2 + (size_t)(c->M + c->N) * 8 + 64;
}

size_t oreduce_tc_smem(const cr_ctx* c) {
    int NCp, NT;
    tc_geometry(c->M, &NCp, &NT);
    return (size_t)NT * 3 * NCp * 32 * 2 + 128 * 32 * 2 + 32 * 8 + 64;
}

// Whether the tensor-core kernels cover this context (M <= 256 and the
// operands fit in shared memory); otherwise the float32 kernels run.
bool tc_supported(const cr_ctx* c) {
    return c->prec == CR_MIXED && c->M <= 256 && ov_tc_smem(c) <= 200 * 1024 &&
           oreduce_tc_smem(c) <= 200 * 1024;
}

cr_status launch_ov_tc(cr_ctx* c, const void* v, const int8_t* spins, int B, const void* T,
                       void* u, const double* skip) {
    int NCp, NT;
    const int cols = tc_geometry(c->M, &NCp, &NT);
    const int Kp = ((c->N + 15) / 16) * 16;
    const size_t sm = ov_tc_smem(c);
    cudaFuncSetAttribute(ov_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const int ntiles = (B + 127) / 128;
    const int grid = ntiles < c->n_sm ? ntiles : c->n_sm;
    CR_LAUNCH(c, CR_KERNEL_OV,
              ov_tc_kernel<<<grid, 128, sm, c->stream>>>(
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
    cudaFuncSetAttribute(oreduce_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    CR_LAUNCH(c, CR_KERNEL_REDUCE,
              oreduce_tc_kernel<<<dim3(nch, (c->N + 127) / 128), 128, sm, c->stream>>>(
                  spins, (const cpx<float>*)T, (const cpx<float>*)g, B, c->N, c->M, c->P, chunk,
                  NCp, NT, cols, c->partial, skip, c->d_status));
    *nch_out = nch;
    return cr_check_launch(c, "oreduce_tc_kernel");
}
