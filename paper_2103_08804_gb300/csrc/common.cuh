// Shared device helpers and the context structure of libchebrbm.
//
// Complex numbers are stored interleaved (re, im); cpx<R> is layout-identical
// to float2 / double2 so that every complex load is one vector load.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "chebrbm.h"

#define CR_HD __host__ __device__ __forceinline__
#define CR_D __device__ __forceinline__

template <typename R>
struct alignas(2 * sizeof(R)) cpx {
    R x, y;
};

template <typename R> CR_HD cpx<R> mk(R x, R y) { return cpx<R>{x, y}; }
template <typename R> CR_HD cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> CR_HD cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> CR_HD cpx<R> operator-(cpx<R> a) { return {-a.x, -a.y}; }
template <typename R> CR_HD cpx<R> operator*(cpx<R> a, cpx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> CR_HD cpx<R> operator*(R s, cpx<R> a) { return {s * a.x, s * a.y}; }
template <typename R> CR_HD cpx<R> conj(cpx<R> a) { return {a.x, -a.y}; }
template <typename R> CR_HD R abs2(cpx<R> a) { return a.x * a.x + a.y * a.y; }
// conj(a) * b
template <typename R> CR_HD cpx<R> cmulc(cpx<R> a, cpx<R> b) {
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename R> CR_HD cpx<R> cdiv(cpx<R> a, cpx<R> b) {
    R d = R(1) / abs2(b);
    return {(a.x * b.x + a.y * b.y) * d, (a.y * b.x - a.x * b.y) * d};
}
template <typename D, typename S> CR_HD cpx<D> ccast(cpx<S> a) { return {(D)a.x, (D)a.y}; }

// Read-only cached complex loads.
CR_D cpx<float> ldg(const cpx<float>* p) {
    float2 v = __ldg((const float2*)p);
    return {v.x, v.y};
}
CR_D cpx<double> ldg(const cpx<double>* p) {
    double2 v = __ldg((const double2*)p);
    return {v.x, v.y};
}

// Math wrappers (CUDA's own functions for each precision).
CR_D float m_exp(float x) { return expf(x); }
CR_D double m_exp(double x) { return exp(x); }
CR_D float m_log1p(float x) { return log1pf(x); }
CR_D double m_log1p(double x) { return log1p(x); }
CR_D float m_atan2(float y, float x) { return atan2f(y, x); }
CR_D double m_atan2(double y, double x) { return atan2(y, x); }
CR_D void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
CR_D void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
CR_D float m_rsqrt(float x) { return rsqrtf(x); }
CR_D double m_rsqrt(double x) { return rsqrt(x); }
CR_D float m_sqrt(float x) { return sqrtf(x); }
CR_D double m_sqrt(double x) { return sqrt(x); }
CR_D float m_cosh(float x) { return coshf(x); }
CR_D double m_cosh(double x) { return cosh(x); }
CR_D float m_sinh(float x) { return sinhf(x); }
CR_D double m_sinh(double x) { return sinh(x); }

template <typename R> CR_D cpx<R> cexp_(cpx<R> z) {
    R e = m_exp(z.x), s, c;
    m_sincos(z.y, &s, &c);
    return {e * c, e * s};
}

// tanh(x + iy) = (sign(x)(1 - e^2) + 2 i e sin 2y) / (1 + e^2 + 2 e cos 2y),
// e = exp(-2|x|): the identity tanh z = sinh 2z-ish form rescaled by e so
// that nothing overflows for large |x|.
template <typename R> CR_D cpx<R> ctanh_(cpx<R> z) {
    R ax = z.x < R(0) ? -z.x : z.x;
    R e = m_exp(R(-2) * ax);
    R e2 = e * e, s, c;
    m_sincos(R(2) * z.y, &s, &c);
    R inv = R(1) / (R(1) + e2 + R(2) * e * c);
    R re = (R(1) - e2) * inv;
    return {z.x < R(0) ? -re : re, R(2) * e * s * inv};
}

// log(2 cosh z) = s z + log(1 + w), s = sign(Re z), w = exp(-2 s z), |w| <= 1.
template <typename R> CR_D cpx<R> clncosh2_(cpx<R> z) {
    R sg = z.x < R(0) ? R(-1) : R(1);
    R e = m_exp(R(-2) * sg * z.x), s, c;
    m_sincos(R(-2) * sg * z.y, &s, &c);
    R wr = e * c, wi = e * s;
    return {sg * z.x + R(0.5) * m_log1p(R(2) * wr + e * e), sg * z.y + m_atan2(wi, R(1) + wr)};
}

// cosh and sinh of a complex number.
template <typename R> CR_D void ccoshsinh_(cpx<R> z, cpx<R>* ch, cpx<R>* sh) {
    R chx = m_cosh(z.x), shx = m_sinh(z.x), s, c;
    m_sincos(z.y, &s, &c);
    *ch = {chx * c, shx * s};
    *sh = {shx * c, chx * s};
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// key bumped by the Weyl constants between rounds.
CR_D uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Warp reductions.
template <typename R> CR_D R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename R> CR_D cpx<R> warp_sum(cpx<R> v) {
    return {warp_sum(v.x), warp_sum(v.y)};
}
template <typename R> CR_D cpx<R> warp_prod(cpx<R> v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cpx<R> w = {__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)};
        v = v * w;
    }
    return v;
}

// Device status codes are cr_status values; the first error wins.
CR_D void set_status(int* st, int code) { atomicCAS(st, 0, code); }

// ------------------------------------------------------------ context

// Bond-ratio tables of one RBM (see rbm.cu, build_tables):
//   D[b][j]  = 2 (W_ij - W_jj')         (b = (i, j'), padded columns 0)
//   Ch[b][j] = cosh D, Sh[b][j] = sinh D (padded columns 1 and 0)
//   ChT/ShT  = the same transposed, [Mp][Nb]
//   ea[b][0] = exp(-2 (a_i - a_j')), ea[b][1] = exp(+2 (a_i - a_j'))
struct cr_tables {
    void* D;
    void* Ch;
    void* Sh;
    void* ChT;
    void* ShT;
    void* ea;
};

struct cr_ktimer {
    int kid;                 // armed kernel family, -1 when off
    int cap, count;
    cudaEvent_t* ev;         // [2 * cap]: start, stop pairs
};

struct cr_ctx {
    int Lx, Ly, N, M, Mp, Nb, P;
    double J;
    cr_prec prec;
    int max_walkers, flags;
    int n_chunks;            // walker chunks of the reductions (<= max_chunks)
    int max_chunks;          // chunks the partial-row workspace holds
    int n_sm;                // multiprocessors of the device
    cudaStream_t stream;
    char err[512];

    int* d_status;           // device status word
    int2* d_bonds;           // [Nb]
    cr_tables tab[2];        // 0: sampler / moment state, 1: target state
    void* theta_tmp;         // [maxB][M]
    void* lp_tmp;            // [2][maxB]
    void* u_tmp;             // [maxB]
    double* partial;         // [n_chunks][P + 2 + M] complex, context precision
    double* red;             // [3][P + 2 + M] complex128 reduced sums
    double* F;               // [P] complex128
    double* cg;              // x, r, p, Ap, diag: [5][P] complex128
    void* p_lo;              // [P] context precision
    double* cgpart;          // per-CTA dot products of a CG step: p.Ap [ceil(P/32)],
                             // r.r and r.z [2][ceil(P/256)]
    double* scal;            // scalars [64]
    double* S;               // [P][P] complex128 (explicit S only)
    void* O_tmp;             // [maxB][P] context precision (explicit S only)
    double* kry;             // Krylov workspace
    size_t kry_len;
    void* Lf;                // [P][P] Cholesky factor, factor precision (blocked path only)
    unsigned char* Xt;       // bf16 hi/lo planes of X^T (mixed explicit S only)
    int2* gtiles;            // lower-triangle blocks of G (mixed explicit S only)
    int n_gtiles;
    // Krylov Gram on the tensor cores (mixed): sized on first use
    unsigned char* gram_x;   // bf16 planes of the B and HB columns
    size_t gram_x_cap;
    double* gram_part;       // per-segment sums
    size_t gram_part_cap;
    int2* gram_tiles;
    size_t gram_tiles_cap;
    int gram_key;            // 2 Nm + (H wanted) of the tile list held, 0 if none
    // estimator sums on the tensor cores (mixed contexts; allocated at creation)
    unsigned char* ored_x;   // bf16 planes of A = [sigma, 1], Y0, Y1
    double* ored_part;       // per-segment sums
    int2* ored_tiles;
    int ored;                // 1 when the path is set up
    void* lp_work;           // linear-prediction scratch (sized on first use)
    size_t lp_work_cap;
    long long n_launches;    // kernels launched so far
    cr_ktimer kt;
    // fused CG solve (cg_fused.cu; mixed contexts with N, M <= 256)
    int fcg;                 // 1 when the fused solve covers this context
    unsigned char* fcg_a1;   // sigma operand tiles of the O v contraction
    unsigned char* fcg_b2;   // sigma^T operand chunks of the O^dag w contraction
    unsigned char* fcg_v2;   // bf16 planes of the W part of p
    size_t fcg_v2plane;
    void* fcg_vab;           // float32 a- and b-parts of p [N + M]
    void* fcg_part;          // partial rows, complex float32 [n_sm][P]
    double* fcg_psc;         // scalar partials [n_sm][8]
    unsigned* fcg_bar;       // grid-barrier counter and abort flag
    int fcg_ctas;            // CTAs of the fused CG (0: one per SM)
    cudaEvent_t ev_fork, ev_join;  // batched runs: fork from / join into the caller's stream
};

static inline int rsize(const cr_ctx* c) { return c->prec == CR_FP64 ? 8 : 4; }

cr_status cr_fail(cr_ctx* c, cr_status s, const char* fmt, ...);
bool cr_kt_begin(cr_ctx* c, int kid);
void cr_kt_end(cr_ctx* c);

// Launch a kernel through the context: counts it and, when its family is
// armed for timing, brackets it with CUDA events on the context stream.
#define CR_LAUNCH(c, kid, ...)                    \
    do {                                          \
        const bool cr_kt_on_ = cr_kt_begin(c, kid); \
        __VA_ARGS__;                              \
        if (cr_kt_on_) cr_kt_end(c);              \
        ++(c)->n_launches;                        \
    } while (0)
#define CR_K_OTHER (-2)
cr_status cr_check_launch(cr_ctx* c, const char* what);

// Explicit S and the direct solve (chol.cu, tc_kernels.cu).  Float64
// contexts up to CHOL_SMALL_P parameters keep the single-CTA float64
// Cholesky; every other explicit-S context takes the blocked path.
#define CHOL_SMALL_P 2048
bool chol_blocked(const cr_ctx* c);
size_t chol_factor_bytes(const cr_ctx* c);
size_t chol_cgpart_len();
cr_status chol_factor(cr_ctx* c);
cr_status chol_refine_solve(cr_ctx* c, const double* F, int maxit);
// Device scratch that grows on demand (once-per-sequence calls only): frees
// and reallocates *p when cap < need; CR_ENOMEM with the caller's name.
cr_status cr_grow(cr_ctx* c, void** p, size_t* cap, size_t need, const char* who);
void ored_sizes(const cr_ctx* c, size_t* x_bytes, size_t* part_bytes, std::vector<int2>* tiles);
cr_status launch_oreduce_tc(cr_ctx* c, const int8_t* spins, const void* T, const void* g, int B,
                            double* redR, double* redO);
cr_status launch_gram_tc(cr_ctx* c, const void* Bm, const void* HBm, int Nm, int B, int ld,
                         double* G, double* H);
cr_status launch_sbuild_tc(cr_ctx* c, const int8_t* spins, const void* T, int B,
                           const double* redO, double shift);
void launch_smirror(cr_ctx* c);  // S[k][l] = conj(S[l][k]) for k < l

// Fused CG solve (cg_fused.cu).
bool fcg_supported(const cr_ctx* c);
void fcg_sizes(const cr_ctx* c, size_t* a1, size_t* b2, size_t* v2plane, size_t* part);
cr_status fcg_prepare(cr_ctx* c);
cr_status launch_cg_fused(cr_ctx* c, const int8_t* spins, const void* T, int B, const double* redO,
                          double shift, double tol, int maxit, int precond, int apply_only,
                          const double* v_in, void* u_out);

// Tables for a state (rbm.cu).
cr_status build_tables(cr_ctx* c, const void* params, int slot);
// theta / log psi of an RBM at a walker batch (rbm.cu).
cr_status launch_logpsi(cr_ctx* c, const void* params, const int8_t* spins, int B, void* theta,
                        void* logpsi);

#define CR_CHECK_ARG(cond, ...)                                  \
    do {                                                         \
        if (!(cond)) return cr_fail(ctx, CR_EINVAL, __VA_ARGS__); \
    } while (0)
