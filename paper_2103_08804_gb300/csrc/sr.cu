// The natural-gradient update of Sec. III on samples of |psi|^2:
//   S_kk' = <O_k* O_k'> - <O_k>* <O_k'>
//   gamma = arccos sqrt(|<R>|^2 / <|R|^2>)
//   F_k   = dgamma gamma cot(gamma) (<O_k* R> / <R> - <O_k*>)
//   (S + lambda I) dalpha = F,  alpha <- alpha + dalpha
// and the VJP of log psi.  O is never stored on the matrix-free path: it is
// rebuilt on the fly from (sigma, tanh theta) with O_a = sigma, O_b = T,
// O_W = sigma (x) T.  Products run in the context precision; every sum over
// walkers is finished in float64 in a fixed order, so results are
// reproducible run to run.
#include "common.cuh"

cr_status launch_ov(cr_ctx* c, const void* v, const int8_t* spins, int B, const void* T, void* u,
                    const double* skip);
bool tc_supported(const cr_ctx* c);
cr_status launch_ov_tc(cr_ctx* c, const void* v, const int8_t* spins, int B, const void* T,
                       void* u, const double* skip);
cr_status launch_oreduce_tc(cr_ctx* c, const int8_t* spins, const void* T, const void* g, int B,
                            const double* skip, int* nch_out);
cr_status logderiv_impl(cr_ctx* ctx, const int8_t* spins, const void* theta, int B, void* tanh_out,
                        void* O_out);

// ------------------------------------------------------------ reductions
//
// partial[c][k] = sum over walker chunk c of op(O_k(s)) g_s, k < P, with
// op = conj or identity, g_s = 1 when g is null; partial[c][P] = sum g_s,
// partial[c][P+1] = sum |g_s|^2; the identity pass (the means Obar) also
// writes partial[c][P+2+j] = sum |T_j(s)|^2, the diagonal of <O* O>.  Rows
// are P + 2 + M long.  Grid (chunk, i-tile): thread t owns hidden units
// j = t + 128 k and the IT visible units of its tile for O_W; CTAs of tile
// 0 also produce the a, b and scalar sums.  FOLD: the sums run in R over
// each block of SUB walkers and are then added into float64 accumulators,
// which bounds the length of every float32 run whatever the chunk length.
template <typename R, int JPT, int IT, bool CONJ, bool FOLD = false>
__global__ void __launch_bounds__(128) oreduce_kernel(const int8_t* __restrict__ spins,
                                                      const cpx<R>* __restrict__ T,
                                                      const cpx<R>* __restrict__ g, int B, int N,
                                                      int M, int P, int chunk,
                                                      double* __restrict__ partial,
                                                      const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;
    constexpr int SUB = 32;
    __shared__ R sg[SUB][IT];
    __shared__ cpx<R> gs[SUB];
    const int c = blockIdx.x, i0 = blockIdx.y * IT, t = threadIdx.x;
    const int s0 = c * chunk, s1 = min(B, s0 + chunk);
    cpx<R> accW[IT][JPT], accb[JPT];
    R acct[JPT];
    // float64 carries of the FOLD form (unused otherwise)
    cpx<double> dW[IT][JPT], db[JPT], da = {0.0, 0.0}, dg = {0.0, 0.0};
    double dt[JPT], dgg = 0.0;
#pragma unroll
    for (int k = 0; k < JPT; ++k) {
        accb[k] = {R(0), R(0)};
        acct[k] = R(0);
        db[k] = {0.0, 0.0};
        dt[k] = 0.0;
#pragma unroll
        for (int ii = 0; ii < IT; ++ii) {
            accW[ii][k] = {R(0), R(0)};
            dW[ii][k] = {0.0, 0.0};
        }
    }
    cpx<R> acca = {R(0), R(0)}, accg = {R(0), R(0)};
    R accgg = R(0);
    // add the float32 block sums into the float64 carries and restart them
    auto fold = [&]() {
#pragma unroll
        for (int k = 0; k < JPT; ++k) {
            db[k] = db[k] + ccast<double>(accb[k]);
            dt[k] += (double)acct[k];
            accb[k] = {R(0), R(0)};
            acct[k] = R(0);
#pragma unroll
            for (int ii = 0; ii < IT; ++ii) {
                dW[ii][k] = dW[ii][k] + ccast<double>(accW[ii][k]);
                accW[ii][k] = {R(0), R(0)};
            }
        }
        da = da + ccast<double>(acca);
        dg = dg + ccast<double>(accg);
        dgg += (double)accgg;
        acca = accg = {R(0), R(0)};
        accgg = R(0);
    };
    for (int sb = s0; sb < s1; sb += SUB) {
        __syncthreads();
        for (int e = t; e < SUB * IT; e += 128) {
            int s = sb + e / IT, i = i0 + e % IT;
            sg[e / IT][e % IT] = (s < s1 && i < N) ? R(spins[(size_t)s * N + i]) : R(0);
        }
        if (t < SUB) {
            int s = sb + t;
            gs[t] = s < s1 ? (g ? g[s] : cpx<R>{R(1), R(0)}) : cpx<R>{R(0), R(0)};
        }
        __syncthreads();
        const int ns = min(SUB, s1 - sb);
        for (int q = 0; q < ns; ++q) {
            const cpx<R> gq = gs[q];
            const int s = sb + q;
#pragma unroll
            for (int k = 0; k < JPT; ++k) {
                int j = t + 128 * k;
                if (j < M) {
                    cpx<R> tv = T[(size_t)s * M + j];
                    if (!CONJ) acct[k] += abs2(tv);
                    if (CONJ) tv = conj(tv);
                    cpx<R> y = tv * gq;
                    accb[k] = accb[k] + y;
#pragma unroll
                    for (int ii = 0; ii < IT; ++ii) {
                        R sv = sg[q][ii];
                        accW[ii][k].x = fma(sv, y.x, accW[ii][k].x);
                        accW[ii][k].y = fma(sv, y.y, accW[ii][k].y);
                    }
                }
            }
            if (t < IT) acca = acca + sg[q][t] * gq;
            if (t == IT) {
                accg = accg + gq;
                accgg += abs2(gq);
            }
        }
        if (FOLD) fold();
    }
    if (!FOLD) fold();  // one carry of the whole chunk
    cpx<double>* out = (cpx<double>*)partial + (size_t)c * (P + 2 + M);
#pragma unroll
    for (int k = 0; k < JPT; ++k) {
        int j = t + 128 * k;
        if (j < M) {
#pragma unroll
            for (int ii = 0; ii < IT; ++ii)
                if (i0 + ii < N) out[N + M + (size_t)(i0 + ii) * M + j] = dW[ii][k];
            if (blockIdx.y == 0) {
                out[N + j] = db[k];
                if (!CONJ) out[P + 2 + j] = {dt[k], 0.0};
            }
        }
    }
    if (t < IT && i0 + t < N) out[i0 + t] = da;
    if (blockIdx.y == 0 && t == IT) {
        out[P] = dg;
        out[P + 1] = {dgg, 0.0};
    }
}

// Compensated (Kahan) accumulation: s + c carries the running sum with the
// low-order part of every addition kept in c (Kahan, CACM 8(1), 1965), so a
// float32 sum over a walker chunk keeps about twice float32's precision.
// The float32 walker sums feed F = c (<O* R>/<R> - <O*>) and S = <O* O> -
// <O*><O>, which cancel when R is nearly constant: plain float32 chunk sums
// left a relative error of ~1e-5 in the moments of a projection step.
template <typename R> CR_D void kadd(R& s, R& c, R v) {
    const R y = v - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
}
template <typename R> CR_D void kadd(cpx<R>& s, cpx<R>& c, cpx<R> v) {
    kadd(s.x, c.x, v.x);
    kadd(s.y, c.y, v.y);
}
// plain or compensated accumulation, chosen at compile time
template <bool COMP, typename R> CR_D void acc_add(cpx<R>& s, cpx<R>& c, cpx<R> v) {
    if constexpr (COMP) kadd(s, c, v);
    else s = s + v;
}
template <bool COMP, typename R> CR_D void acc_add(R& s, R& c, R v) {
    if constexpr (COMP) kadd(s, c, v);
    else s += v;
}

// Register-tiled form of the same reduction (used by the hot path).  Each CTA
// of 128 threads takes a walker chunk and a tile of 64 visible x 32 hidden
// units; thread t owns visible units i0 + 4 (t / 8) + {0..3} and hidden units
// j0 + 4 (t % 8) + {0..3}, so each staged step feeds 32 FMAs from 3 shared
// loads.  Y_sj = op(T_sj) g_s is formed once per walker while staging, and
// the next sub-block's T and spins are fetched into registers while the
// current one is consumed.  Partial rows and their layout are those of
// oreduce_kernel.  COMP: Kahan-compensated sums (the estimators of F, Obar
// and the VJP); plain sums for the CG products of the float32 path.
template <typename R, bool CONJ, bool COMP = false>
__global__ void __launch_bounds__(128) oreduce2_kernel(const int8_t* __restrict__ spins,
                                                       const cpx<R>* __restrict__ T,
                                                       const cpx<R>* __restrict__ g, int B, int N,
                                                       int M, int P, int chunk,
                                                       double* __restrict__ partial,
                                                       const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;
    constexpr int SUB = 32, TI = 64, TJ = 32, NT = 128;
    constexpr int SE = SUB * TI / NT, YE = SUB * TJ / NT;   // staged elements per thread
    __shared__ __align__(16) R sg[SUB][TI];
    __shared__ __align__(16) cpx<R> ys[SUB][TJ];
    __shared__ cpx<R> gs[SUB];
    const int c = blockIdx.x, j0 = blockIdx.y * TJ, i0 = blockIdx.z * TI;
    const int t = threadIdx.x, ti = 4 * (t >> 3), tj = 4 * (t & 7);
    const int s0 = c * chunk, s1 = min(B, s0 + chunk);
    const bool a_cta = blockIdx.y == 0, b_cta = blockIdx.z == 0;
    cpx<R> acc[4][4], accb[4];
    R acct[4];
    // compensation terms (unused, and removed by the compiler, when !COMP)
    cpx<R> cmp[4][4], cmpb[4];
    R cmpt[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][k] = cmp[a][k] = {R(0), R(0)};
        accb[k] = cmpb[k] = {R(0), R(0)};
        acct[k] = cmpt[k] = R(0);
    }
    cpx<R> acca = {R(0), R(0)}, accg = {R(0), R(0)}, cmpa = {R(0), R(0)}, cmpg = {R(0), R(0)};
    R accgg = R(0), cmpgg = R(0);
    // register prefetch of one sub-block
    int8_t sp[SE];
    cpx<R> tp[YE];
    auto fetch = [&](int sb) {
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            const int e = t + u * NT, w = e / TI, i = e % TI, s = sb + w;
            sp[u] = (s < s1 && i0 + i < N) ? spins[(size_t)s * N + i0 + i] : (int8_t)0;
        }
#pragma unroll
        for (int u = 0; u < YE; ++u) {
            const int e = t + u * NT, w = e / TJ, j = e % TJ, s = sb + w;
            tp[u] = (s < s1 && j0 + j < M) ? T[(size_t)s * M + j0 + j] : cpx<R>{R(0), R(0)};
        }
    };
    if (s0 < s1) fetch(s0);
    for (int sb = s0; sb < s1; sb += SUB) {
        __syncthreads();
        if (t < SUB) {
            const int s = sb + t;
            gs[t] = s < s1 ? (g ? g[s] : cpx<R>{R(1), R(0)}) : cpx<R>{R(0), R(0)};
        }
#pragma unroll
        for (int u = 0; u < SE; ++u) {
            const int e = t + u * NT;
            sg[e / TI][e % TI] = R(sp[u]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < YE; ++u) {
            const int e = t + u * NT, w = e / TJ;
            cpx<R> tv = tp[u];
            if (CONJ) tv = conj(tv);
            ys[w][e % TJ] = tv * gs[w];
        }
        if (sb + SUB < s1) fetch(sb + SUB);
        __syncthreads();
        const int ns = min(SUB, s1 - sb);
        for (int q = 0; q < ns; ++q) {
            R sv[4];
            cpx<R> y[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) sv[a] = sg[q][ti + a];
#pragma unroll
            for (int k = 0; k < 4; ++k) y[k] = ys[q][tj + k];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if constexpr (COMP) {
                        kadd(acc[a][k], cmp[a][k], sv[a] * y[k]);  // sigma = +-1, 0: exact
                    } else {
                        acc[a][k].x = fma(sv[a], y[k].x, acc[a][k].x);
                        acc[a][k].y = fma(sv[a], y[k].y, acc[a][k].y);
                    }
                }
            if (ti == 0) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    acc_add<COMP>(accb[k], cmpb[k], y[k]);
                    if (!CONJ) acc_add<COMP>(acct[k], cmpt[k], abs2(y[k]));
                }
            }
            if (a_cta && t < TI) acc_add<COMP>(acca, cmpa, sg[q][t] * gs[q]);
            if (t == 0) {
                acc_add<COMP>(accg, cmpg, gs[q]);
                acc_add<COMP>(accgg, cmpgg, abs2(gs[q]));
            }
        }
    }
    // partial rows in the context precision (the sums above are in R); a
    // compensated sum is s - c (c holds the excess of s)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a][k] = acc[a][k] - cmp[a][k];
        accb[k] = accb[k] - cmpb[k];
        acct[k] -= cmpt[k];
    }
    acca = acca - cmpa;
    accg = accg - cmpg;
    accgg -= cmpgg;
    cpx<R>* out = (cpx<R>*)partial + (size_t)c * (P + 2 + M);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int j = j0 + tj + k;
        if (j >= M) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + ti + a;
            if (i < N) out[N + M + (size_t)i * M + j] = acc[a][k];
        }
        if (b_cta && ti == 0) {
            out[N + j] = accb[k];
            if (!CONJ) out[P + 2 + j] = {acct[k], R(0)};
        }
    }
    if (a_cta && t < TI && i0 + t < N) out[i0 + t] = acca;
    if (a_cta && b_cta && t == 0) {
        out[P] = accg;
        out[P + 1] = {accgg, R(0)};
    }
}

// red[k] = sum over chunks of partial[c][k] (k < len, rows `stride` long of
// cpx<RP>), in chunk order, in float64.
template <typename RP>
__global__ void combine_kernel(const double* __restrict__ partial, int n_chunks, int len,
                               int stride, double* __restrict__ red,
                               const double* __restrict__ skip) {
    if (skip && *skip != 0.0) return;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= len) return;
    const cpx<RP>* p = (const cpx<RP>*)partial;
    cpx<double> s = {0.0, 0.0};
    for (int c = 0; c < n_chunks; ++c) s = s + ccast<double>(p[(size_t)c * stride + k]);
    ((cpx<double>*)red)[k] = s;
}

template <typename R, bool CONJ, bool COMP>
static cr_status oreduce_t(cr_ctx* c, const int8_t* spins, const void* T, const void* g, int B,
                           double* red_out, const double* skip) {
    const int N = c->N, M = c->M, P = c->P;
    const int nch = c->n_chunks < B ? c->n_chunks : B;
    const int chunk = (B + nch - 1) / nch;
    CR_LAUNCH(c, CR_KERNEL_REDUCE,
              (oreduce2_kernel<R, CONJ, COMP><<<dim3(nch, (M + 31) / 32, (N + 63) / 64), 128, 0,
                                                c->stream>>>(spins, (const cpx<R>*)T,
                                                             (const cpx<R>*)g, B, N, M, P, chunk,
                                                             c->partial, skip)));
    cr_status s = cr_check_launch(c, "oreduce2_kernel");
    if (s != CR_OK) return s;
    if (!red_out) return CR_OK;  // the caller combines the chunk rows itself
    const int len = CONJ ? P + 2 : P + 2 + M;
    CR_LAUNCH(c, CR_K_OTHER, combine_kernel<R><<<(len + 255) / 256, 256, 0, c->stream>>>(
                                 c->partial, nch, len, P + 2 + M, red_out, skip));
    return cr_check_launch(c, "combine_kernel");
}

// comp: compensated float32 sums (estimators and the VJP); float64 contexts
// sum plainly in float64.
static cr_status oreduce(cr_ctx* c, bool conj_, const int8_t* spins, const void* T, const void* g,
                         int B, double* red_out, const double* skip, bool comp = true) {
    if (c->prec == CR_FP64)
        return conj_ ? oreduce_t<double, true, false>(c, spins, T, g, B, red_out, skip)
                     : oreduce_t<double, false, false>(c, spins, T, g, B, red_out, skip);
    if (comp)
        return conj_ ? oreduce_t<float, true, true>(c, spins, T, g, B, red_out, skip)
                     : oreduce_t<float, false, true>(c, spins, T, g, B, red_out, skip);
    return conj_ ? oreduce_t<float, true, false>(c, spins, T, g, B, red_out, skip)
                 : oreduce_t<float, false, false>(c, spins, T, g, B, red_out, skip);
}

// ----------------------------------------------------------------- force
//
// From redR = [sum conj(O) R | sum R | sum |R|^2] and redO = [sum O | ...]:
// <R>, <|R|^2>, gamma (argument clamped to <= 1), c = dgamma gamma cot gamma
// (1 below 1e-8), F_k = c (<O_k* R>/<R> - conj(<O_k>)).
__device__ void force_scalars(const cpx<double>* redR, int P, int B, double dgamma, cpx<double>* mR,
                              double* mRR, double* gamma, double* cc) {
    const double inv = 1.0 / B;
    *mR = inv * redR[P];
    *mRR = redR[P + 1].x * inv;
    double ratio = abs2(*mR) / *mRR;
    if (!(ratio <= 1.0)) ratio = ratio > 1.0 ? 1.0 : ratio;
    *gamma = acos(sqrt(ratio));
    *cc = dgamma * (*gamma < 1e-8 ? 1.0 : *gamma / tan(*gamma));
}

// mode CR_SR_FIT: F = dgamma gamma cot gamma (<O* R>/<R> - <O*>) (Sec. III);
// mode CR_SR_ENERGY: F = -dgamma (<O* R> - <O*> <R>), R the local energy.
__global__ void force_kernel(const double* __restrict__ redR_, const double* __restrict__ redO_,
                             int P, int B, double dgamma, int mode, double* __restrict__ F_,
                             double* __restrict__ stats, int* __restrict__ status) {
    const cpx<double>* redR = (const cpx<double>*)redR_;
    const cpx<double>* redO = (const cpx<double>*)redO_;
    cpx<double> mR;
    double mRR, gamma, cc;
    force_scalars(redR, P, B, dgamma, &mR, &mRR, &gamma, &cc);
    const double inv = 1.0 / B;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        cpx<double> f;
        if (mode == CR_SR_ENERGY)
            f = -dgamma * (inv * redR[k] - conj(inv * redO[k]) * mR);
        else
            f = cc * (cdiv(inv * redR[k], mR) - conj(inv * redO[k]));
        ((cpx<double>*)F_)[k] = f;
    }
    if (k == 0) {
        const bool bad = !isfinite(mR.x) || !isfinite(mR.y) || !isfinite(mRR) ||
                         (mode != CR_SR_ENERGY && abs2(mR) == 0.0);
        if (bad) set_status(status, CR_ENONFINITE);
        if (stats) {
            stats[0] = mode == CR_SR_ENERGY ? 0.0 : gamma;
            stats[1] = mR.x;
            stats[2] = mR.y;
            stats[3] = mRR;
            stats[4] = cc;
        }
    }
}

// ------------------------------------------------------ explicit S (small P)

template <typename R>
__global__ void o_from_tanh_kernel(const int8_t* __restrict__ spins, const cpx<R>* __restrict__ T,
                                   int B, int N, int M, int P, cpx<R>* __restrict__ O) {
    size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (size_t)B * P) return;
    int s = (int)(idx / P), k = (int)(idx % P);
    cpx<R> v;
    if (k < N) v = {R(spins[(size_t)s * N + k]), R(0)};
    else if (k < N + M) v = T[(size_t)s * M + (k - N)];
    else {
        int i = (k - N - M) / M, j = (k - N - M) % M;
        v = R(spins[(size_t)s * N + i]) * T[(size_t)s * M + j];
    }
    O[idx] = v;
}

// S[k][l] = sum_s conj(O_sk) O_sl / B - conj(Obar_k) Obar_l + shift delta_kl, float64.
template <typename R>
__global__ void sbuild_kernel(const cpx<R>* __restrict__ O, int B, int P,
                              const double* __restrict__ redO_, double shift,
                              double* __restrict__ S_) {
    __shared__ cpx<R> tk[16][17], tl[16][17];
    const int k = blockIdx.y * 16 + threadIdx.y, l = blockIdx.x * 16 + threadIdx.x;
    cpx<double> acc = {0.0, 0.0};
    for (int s0 = 0; s0 < B; s0 += 16) {
        int s = s0 + threadIdx.x;
        int kk = blockIdx.y * 16 + threadIdx.y;
        tk[threadIdx.y][threadIdx.x] = (s < B && kk < P) ? O[(size_t)s * P + kk] : cpx<R>{R(0), R(0)};
        s = s0 + threadIdx.y;
        tl[threadIdx.y][threadIdx.x] = (s < B && l < P) ? O[(size_t)s * P + l] : cpx<R>{R(0), R(0)};
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q)
            acc = acc + ccast<double>(cmulc(tk[threadIdx.y][q], tl[q][threadIdx.x]));
        __syncthreads();
    }
    if (k < P && l < P) {
        const cpx<double>* redO = (const cpx<double>*)redO_;
        const double inv = 1.0 / B;
        cpx<double> v = inv * acc - cmulc(inv * redO[k], inv * redO[l]);
        if (k == l) v.x += shift;
        ((cpx<double>*)S_)[(size_t)k * P + l] = v;
    }
}

// In-place Cholesky S = L L^dag (lower triangle), one CTA, then
// L y = F, L^dag x = y; x written to out.  Column-oriented so each step is
// one parallel update and one barrier.
__global__ void __launch_bounds__(1024) chol_solve_kernel(double* __restrict__ S_, int P,
                                                          const double* __restrict__ F_,
                                                          double* __restrict__ x_,
                                                          int* __restrict__ status) {
    cpx<double>* S = (cpx<double>*)S_;
    cpx<double>* x = (cpx<double>*)x_;
    const cpx<double>* F = (const cpx<double>*)F_;
    __shared__ double piv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    // right-looking factorisation
    for (int j = 0; j < P; ++j) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double d = S[(size_t)j * P + j].x;
            if (!(d > 0.0)) {
                bad = 1;
                d = 1.0;
            }
            piv = sqrt(d);
            S[(size_t)j * P + j] = {piv, 0.0};
        }
        __syncthreads();
        const double ip = 1.0 / piv;
        for (int i = j + 1 + threadIdx.x; i < P; i += blockDim.x)
            S[(size_t)i * P + j] = ip * S[(size_t)i * P + j];
        __syncthreads();
        // trailing update of the lower triangle: S_il -= L_ij conj(L_lj), l <= i
        const int n = P - j - 1;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            int i = j + 1 + e / n, l = j + 1 + e % n;
            if (l <= i) S[(size_t)i * P + l] = S[(size_t)i * P + l] -
                                               S[(size_t)i * P + j] * conj(S[(size_t)l * P + j]);
        }
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) set_status(status, CR_ESINGULAR);
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x) x[i] = F[i];
    // forward: L y = F
    for (int k = 0; k < P; ++k) {
        __syncthreads();
        cpx<double> yk = (1.0 / S[(size_t)k * P + k].x) * x[k];
        __syncthreads();
        if (threadIdx.x == 0) x[k] = yk;
        for (int i = k + 1 + threadIdx.x; i < P; i += blockDim.x)
            x[i] = x[i] - S[(size_t)i * P + k] * yk;
    }
    // backward: L^dag x = y
    for (int k = P - 1; k >= 0; --k) {
        __syncthreads();
        cpx<double> xk = (1.0 / S[(size_t)k * P + k].x) * x[k];
        __syncthreads();
        if (threadIdx.x == 0) x[k] = xk;
        for (int i = threadIdx.x; i < k; i += blockDim.x)
            x[i] = x[i] - conj(S[(size_t)k * P + i]) * xk;
    }
}

// ------------------------------------------------------------------- CG
//
// Matrix-free S v = (O^dag (O v) - conj(Obar) sum_s (O v)_s) / B, using
// sum_s (O_s - Obar) = 0.  Conjugate gradients from x = 0 (Hestenes and
// Stiefel), optionally preconditioned with d = diag(S) + shift, where
// S_kk = <|O_k|^2> - |Obar_k|^2 with |O_a|^2 = 1 and |O_b|^2 = |O_W|^2 =
// |T_j|^2.  Vectors x, r, p, Ap, d and all scalars in float64; the
// O-products run in the context precision.  scal: [0] r.z, [1] F.F,
// [2] done flag, [3] iterations, [4] r.r.

__device__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

template <typename R>
__global__ void __launch_bounds__(1024) cg_init_kernel(const double* __restrict__ F_,
                                                       const double* __restrict__ redO_, int N,
                                                       int M, int P, int B, double shift,
                                                       int precond, double* __restrict__ cg_,
                                                       cpx<R>* __restrict__ p_lo,
                                                       double* __restrict__ scal) {
    __shared__ double red[32];
    const cpx<double>* F = (const cpx<double>*)F_;
    const cpx<double>* sO = (const cpx<double>*)redO_;
    cpx<double>* x = (cpx<double>*)cg_;
    cpx<double>* r = x + P;
    cpx<double>* p = x + 2 * P;
    cpx<double>* dg = x + 4 * P;
    const double inv = 1.0 / B;
    double ff = 0.0, rz = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) {
        double d = 1.0;
        if (precond) {
            double o2 = k < N ? 1.0 : inv * sO[P + 2 + (k < N + M ? k - N : (k - N - M) % M)].x;
            d = o2 - abs2(inv * sO[k]) + shift;
        }
        cpx<double> f = F[k];
        cpx<double> z = (1.0 / d) * f;
        x[k] = {0.0, 0.0};
        r[k] = f;
        p[k] = z;
        dg[k] = {d, 0.0};
        p_lo[k] = ccast<R>(z);
        ff += abs2(f);
        rz += cmulc(f, z).x;
    }
    ff = block_sum(ff, red);
    rz = block_sum(rz, red);
    if (threadIdx.x == 0) {
        scal[5] = rz;
        scal[1] = ff;
        scal[2] = ff == 0.0 ? 1.0 : 0.0;
        scal[3] = 0.0;
        scal[4] = ff;
    }
}

// Multi-CTA CG step, three launches per iteration.  scal[5 + (it & 1)]
// holds r.z of iteration it, so the last kernel writes the next value into
// the other slot while its CTAs still read the current one.  Per-CTA partial
// dot products go to part[3][nblk] and are summed by every CTA in the same
// fixed order (deterministic).
constexpr int CG_TPB = 256;

__device__ double sum_parts(const double* p, int n, double* red) {
    double v = 0.0;
    for (int b = threadIdx.x; b < n; b += blockDim.x) v += p[b];
    return block_sum(v, red);
}

// Ap = S p + shift p from the chunk rows of sum conj(O) (O p) (the combine
// fused in), and the per-CTA share of p.Ap.  A CTA takes 32 parameters; its
// 8 warps each sum every 8th chunk row, then warp 0 adds the 8 group sums in
// order (a fixed summation order, so the result is deterministic).
constexpr int CGA_K = 32;

template <typename RP>
__global__ void __launch_bounds__(256) cg_apply_kernel(const double* __restrict__ partial,
                                                       int nch, int stride,
                                                       const double* __restrict__ redO_, int P,
                                                       int B, double shift,
                                                       double* __restrict__ cg_,
                                                       double* __restrict__ part,
                                                       const double* __restrict__ scal) {
    if (scal[2] != 0.0) return;
    __shared__ cpx<double> grp[8][CGA_K];
    __shared__ cpx<double> smu;
    const cpx<RP>* pt = (const cpx<RP>*)partial;
    const cpx<double>* sO = (const cpx<double>*)redO_;
    cpx<double>* p = (cpx<double>*)cg_ + 2 * P;
    cpx<double>* Ap = (cpx<double>*)cg_ + 3 * P;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int k = blockIdx.x * CGA_K + lane;
    cpx<double> w = {0.0, 0.0};
    if (k < P)
        for (int c = wid; c < nch; c += 8) w = w + ccast<double>(pt[(size_t)c * stride + k]);
    grp[wid][lane] = w;
    if (wid == 7) {
        cpx<double> su = {0.0, 0.0};
        for (int c = lane; c < nch; c += 32) su = su + ccast<double>(pt[(size_t)c * stride + P]);
        su = warp_sum(su);
        if (lane == 0) smu = su;
    }
    __syncthreads();
    if (wid == 0) {
        const double inv = 1.0 / B;
        double pap = 0.0;
        if (k < P) {
            cpx<double> tot = grp[0][lane];
#pragma unroll
            for (int gi = 1; gi < 8; ++gi) tot = tot + grp[gi][lane];
            cpx<double> a = inv * tot - conj(inv * sO[k]) * (inv * smu) + shift * p[k];
            Ap[k] = a;
            pap = cmulc(p[k], a).x;
        }
        pap = warp_sum(pap);
        if (lane == 0) part[blockIdx.x] = pap;
    }
}

// alpha = r.z / p.Ap; x += alpha p; r -= alpha Ap; shares of r.r and r.z.
__global__ void __launch_bounds__(CG_TPB) cg_xr_kernel(int P, double* __restrict__ cg_,
                                                       double* __restrict__ part, int napp,
                                                       int nblk, const double* __restrict__ scal,
                                                       int slot) {
    if (scal[2] != 0.0) return;
    __shared__ double red[32];
    cpx<double>* x = (cpx<double>*)cg_;
    cpx<double>* r = x + P;
    const cpx<double>* p = x + 2 * P;
    const cpx<double>* Ap = x + 3 * P;
    const cpx<double>* dg = x + 4 * P;
    const double alpha = scal[5 + slot] / sum_parts(part, napp, red);
    part += napp;  // this kernel's shares follow the p.Ap shares
    const int k = blockIdx.x * CG_TPB + threadIdx.x;
    double rn = 0.0, rz = 0.0;
    if (k < P) {
        x[k] = x[k] + alpha * p[k];
        cpx<double> rk = r[k] - alpha * Ap[k];
        r[k] = rk;
        rn = abs2(rk);
        rz = (1.0 / dg[k].x) * rn;
    }
    rn = block_sum(rn, red);
    rz = block_sum(rz, red);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = rn;
        part[nblk + blockIdx.x] = rz;
    }
}

// Convergence test |r| <= tol |F|, then beta = r.z(new) / r.z and p = z + beta p.
template <typename R>
__global__ void __launch_bounds__(CG_TPB) cg_p_kernel(int P, double tol, double* __restrict__ cg_,
                                                      cpx<R>* __restrict__ p_lo,
                                                      double* __restrict__ part, int nblk,
                                                      double* __restrict__ scal, int slot) {
    if (scal[2] != 0.0) return;
    __shared__ double red[32];
    const cpx<double>* r = (const cpx<double>*)cg_ + P;
    cpx<double>* p = (cpx<double>*)cg_ + 2 * P;
    const cpx<double>* dg = (const cpx<double>*)cg_ + 4 * P;
    const double rn = sum_parts(part, nblk, red);
    const double rzn = sum_parts(part + nblk, nblk, red);
    const bool done = !(rn > tol * tol * scal[1]);
    const int k = blockIdx.x * CG_TPB + threadIdx.x;
    if (!done && k < P) {
        const double beta = rzn / scal[5 + slot];
        cpx<double> pk = (1.0 / dg[k].x) * r[k] + beta * p[k];
        p[k] = pk;
        p_lo[k] = ccast<R>(pk);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        scal[5 + (slot ^ 1)] = rzn;
        scal[3] += 1.0;
        scal[4] = rn;
        if (done) scal[2] = 1.0;
    }
}

// strict: CG that ended at its iteration limit above tolerance (done flag
// scal[2] unset) reports CR_ENOTCONV in the device status word.
template <typename R>
__global__ void apply_update_kernel(cpx<R>* __restrict__ prm, const double* __restrict__ x_, int P,
                                    const double* __restrict__ scal, double* __restrict__ stats,
                                    const double* __restrict__ F_, int* __restrict__ status,
                                    int cg, int strict) {
    const cpx<double>* x = (const cpx<double>*)x_;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        cpx<double> v = ccast<double>(prm[k]) + x[k];
        if (!isfinite(v.x) || !isfinite(v.y)) set_status(status, CR_ENONFINITE);
        prm[k] = ccast<R>(v);
    }
    if (k == 0 && strict && scal[2] == 0.0) set_status(status, CR_ENOTCONV);
    if (k == 0 && stats) {
        stats[5] = cg ? scal[3] : 0.0;
        stats[6] = cg ? (scal[1] > 0 ? sqrt(scal[4] / scal[1]) : 0.0) : 0.0;
        stats[7] = sqrt(scal[1]);
    }
}

__global__ void fnorm_kernel(const double* __restrict__ F_, int P, double* __restrict__ scal) {
    __shared__ double red[32];
    const cpx<double>* F = (const cpx<double>*)F_;
    double s = 0.0;
    for (int k = threadIdx.x; k < P; k += blockDim.x) s += abs2(F[k]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) scal[1] = s;
}

// S + shift I into c->S (full Hermitian, float64; the upper triangle a
// mirror of the lower): tensor cores (bf16x3) for mixed contexts; otherwise
// O materialised in the context precision and its Gram matrix accumulated
// in float64.
template <typename R>
static cr_status build_s(cr_ctx* c, const int8_t* spins, const void* T, int B,
                         const double* redO, double shift) {
    if (c->prec == CR_MIXED) return launch_sbuild_tc(c, spins, T, B, redO, shift);
    const int P = c->P;
    const size_t n = (size_t)B * P;
    CR_LAUNCH(c, CR_K_OTHER,
              o_from_tanh_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(
                  spins, (const cpx<R>*)T, B, c->N, c->M, P, (cpx<R>*)c->O_tmp));
    dim3 g((P + 15) / 16, (P + 15) / 16);
    CR_LAUNCH(c, CR_KERNEL_SBUILD,
              sbuild_kernel<R><<<g, dim3(16, 16), 0, c->stream>>>((const cpx<R>*)c->O_tmp, B, P,
                                                                  redO, shift, c->S));
    launch_smirror(c);  // exactly Hermitian off the diagonal
    return cr_check_launch(c, "explicit S");
}

template <typename R>
static cr_status sr_step_t(cr_ctx* c, void* params, const int8_t* spins, const void* T,
                           const void* Rv, int B, const cr_sr_opts* o, double* stats) {
    const int P = c->P;
    double* redR = c->red;
    double* redO = c->red + 2 * (P + 2 + c->M);
    cr_status s;
    if (c->ored && o->solver == CR_SOLVE_CG && !o->cg_precond) {
        // mixed, matrix-free CG: both estimator sums in one tensor-core launch
        // (about 3e-7 of the summed terms).  The direct solve of an explicit S
        // keeps the compensated float32 sums (about 1e-8): it solves at the
        // small shift exactly, with no CG budget to damp their error.
        s = launch_oreduce_tc(c, spins, T, Rv, B, redR, redO);
    } else {
        s = oreduce(c, true, spins, T, Rv, B, redR, nullptr);
        if (s == CR_OK) s = oreduce(c, false, spins, T, nullptr, B, redO, nullptr);
    }
    if (s != CR_OK) return s;
    CR_LAUNCH(c, CR_K_OTHER, force_kernel<<<(P + 255) / 256, 256, 0, c->stream>>>(
                                 redR, redO, P, B, o->dgamma, o->mode, c->F, stats, c->d_status));
    if ((s = cr_check_launch(c, "force_kernel")) != CR_OK) return s;
    double* x = c->cg;
    const bool blocked = o->solver == CR_SOLVE_CHOLESKY && chol_blocked(c);
    if (o->solver == CR_SOLVE_CHOLESKY) {
        if ((s = build_s<R>(c, spins, T, B, redO, o->shift)) != CR_OK) return s;
        if (blocked) {
            if ((s = chol_factor(c)) != CR_OK) return s;
            if ((s = chol_refine_solve(c, c->F, o->cg_maxit)) != CR_OK) return s;
        } else {
            CR_LAUNCH(c, CR_K_OTHER, chol_solve_kernel<<<1, 1024, 0, c->stream>>>(c->S, P, c->F, x, c->d_status));
            CR_LAUNCH(c, CR_K_OTHER, fnorm_kernel<<<1, 1024, 0, c->stream>>>(c->F, P, c->scal));
            if ((s = cr_check_launch(c, "cholesky path")) != CR_OK) return s;
        }
    } else if (c->fcg) {
        // mixed precision: the whole CG in one persistent tensor-core kernel
        s = launch_cg_fused(c, spins, T, B, redO, o->shift, o->cg_tol, o->cg_maxit, o->cg_precond,
                            0, nullptr, nullptr);
        if (s != CR_OK) return s;
    } else {
        CR_LAUNCH(c, CR_K_OTHER, cg_init_kernel<R><<<1, 1024, 0, c->stream>>>(
                                     c->F, redO, c->N, c->M, P, B, o->shift, o->cg_precond,
                                     c->cg, (cpx<R>*)c->p_lo, c->scal));
        if ((s = cr_check_launch(c, "cg_init")) != CR_OK) return s;
        const double* done = c->scal + 2;
        const int nblk = (P + CG_TPB - 1) / CG_TPB;
        const int napp = (P + CGA_K - 1) / CGA_K;
        const bool tcp = tc_supported(c);  // mixed precision: tensor-core products
        int nch = c->n_chunks < B ? c->n_chunks : B;
        for (int it = 0; it < o->cg_maxit; ++it) {
            if (tcp) {
                s = launch_ov_tc(c, c->p_lo, spins, B, T, c->u_tmp, done);
                if (s != CR_OK) return s;
                s = launch_oreduce_tc(c, spins, T, c->u_tmp, B, done, &nch);
            } else {
                s = launch_ov(c, c->p_lo, spins, B, T, c->u_tmp, done);
                if (s != CR_OK) return s;
                s = oreduce(c, true, spins, T, c->u_tmp, B, nullptr, done, false);
            }
            if (s != CR_OK) return s;
            CR_LAUNCH(c, CR_KERNEL_CG, cg_apply_kernel<R><<<napp, 256, 0, c->stream>>>(
                                           c->partial, nch, P + 2 + c->M, redO, P, B, o->shift,
                                           c->cg, c->cgpart, c->scal));
            CR_LAUNCH(c, CR_KERNEL_CG, cg_xr_kernel<<<nblk, CG_TPB, 0, c->stream>>>(
                                           P, c->cg, c->cgpart, napp, nblk, c->scal, it & 1));
            CR_LAUNCH(c, CR_KERNEL_CG, cg_p_kernel<R><<<nblk, CG_TPB, 0, c->stream>>>(
                                           P, o->cg_tol, c->cg, (cpx<R>*)c->p_lo,
                                           c->cgpart + napp, nblk, c->scal, it & 1));
            if ((s = cr_check_launch(c, "cg step")) != CR_OK) return s;
        }
    }
    CR_LAUNCH(c, CR_K_OTHER, apply_update_kernel<R><<<(P + 255) / 256, 256, 0, c->stream>>>(
        (cpx<R>*)params, x, P, c->scal, stats, c->F, c->d_status, o->solver == CR_SOLVE_CG || blocked,
        o->solver == CR_SOLVE_CG && o->cg_strict));
    return cr_check_launch(c, "apply_update");
}

extern "C" cr_status sr_step(cr_ctx* ctx, void* params, const int8_t* spins, const void* tanh_theta,
                             const void* R, int B, const cr_sr_opts* opts, double* stats_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(params && opts, "sr_step: null params or opts");
    CR_CHECK_ARG(B >= 1 && B <= ctx->max_walkers, "sr_step: B=%d outside [1, %d]", B,
                 ctx->max_walkers);
    CR_CHECK_ARG(spins && tanh_theta && R, "sr_step: null array");
    CR_CHECK_ARG(opts->shift >= 0.0, "sr_step: shift must be >= 0");
    CR_CHECK_ARG(opts->solver == CR_SOLVE_CHOLESKY || opts->solver == CR_SOLVE_CG,
                 "sr_step: unknown solver");
    CR_CHECK_ARG(opts->solver != CR_SOLVE_CHOLESKY || (ctx->flags & CR_CTX_EXPLICIT_S),
                 "sr_step: Cholesky needs a context created with CR_CTX_EXPLICIT_S");
    CR_CHECK_ARG(opts->mode == CR_SR_FIT || opts->mode == CR_SR_ENERGY, "sr_step: unknown mode");
    CR_CHECK_ARG(opts->solver != CR_SOLVE_CG || (opts->cg_maxit >= 1 && opts->cg_tol >= 0.0 &&
                                                 (opts->cg_precond == 0 || opts->cg_precond == 1)),
                 "sr_step: bad CG options");
    CR_CHECK_ARG(opts->cg_strict == 0 || opts->cg_strict == 1, "sr_step: cg_strict must be 0 or 1");
    return ctx->prec == CR_FP64
               ? sr_step_t<double>(ctx, params, spins, tanh_theta, R, B, opts, stats_out)
               : sr_step_t<float>(ctx, params, spins, tanh_theta, R, B, opts, stats_out);
}

// v (complex128) into the CG direction p (float64) and its context-precision
// copy, with the done flag cleared, so that one CG product runs on it.
template <typename R>
__global__ void sv_load_kernel(const double* __restrict__ v_, int P, double* __restrict__ cg_,
                               cpx<R>* __restrict__ p_lo, double* __restrict__ scal) {
    const cpx<double>* v = (const cpx<double>*)v_;
    cpx<double>* p = (cpx<double>*)cg_ + 2 * P;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) {
        p[k] = v[k];
        p_lo[k] = ccast<R>(v[k]);
    }
    if (k == 0) scal[2] = 0.0;
}

template <typename R>
static cr_status sv_t(cr_ctx* c, const int8_t* spins, const void* T, int B, const double* v,
                      double shift, void* u_out, double* out) {
    const int P = c->P;
    double* redO = c->red + 2 * (P + 2 + c->M);
    cr_status s = oreduce(c, false, spins, T, nullptr, B, redO, nullptr);
    if (s != CR_OK) return s;
    if (c->fcg) {
        s = launch_cg_fused(c, spins, T, B, redO, shift, 0.0, 1, 0, 1, v, u_out);
        if (s != CR_OK) return s;
        cudaError_t e = cudaMemcpyAsync(out, c->cg + 6 * (size_t)P, (size_t)P * 16,
                                        cudaMemcpyDeviceToDevice, c->stream);
        return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "sr_sv copy: %s", cudaGetErrorString(e));
    }
    CR_LAUNCH(c, CR_K_OTHER, sv_load_kernel<R><<<(P + 255) / 256, 256, 0, c->stream>>>(
                                 v, P, c->cg, (cpx<R>*)c->p_lo, c->scal));
    if ((s = cr_check_launch(c, "sv_load")) != CR_OK) return s;
    const double* done = c->scal + 2;
    int nch = c->n_chunks < B ? c->n_chunks : B;
    if (tc_supported(c)) {
        if ((s = launch_ov_tc(c, c->p_lo, spins, B, T, c->u_tmp, done)) != CR_OK) return s;
        s = launch_oreduce_tc(c, spins, T, c->u_tmp, B, done, &nch);
    } else {
        if ((s = launch_ov(c, c->p_lo, spins, B, T, c->u_tmp, done)) != CR_OK) return s;
        s = oreduce(c, true, spins, T, c->u_tmp, B, nullptr, done, false);
    }
    if (s != CR_OK) return s;
    const int napp = (P + CGA_K - 1) / CGA_K;
    CR_LAUNCH(c, CR_KERNEL_CG, cg_apply_kernel<R><<<napp, 256, 0, c->stream>>>(
                                   c->partial, nch, P + 2 + c->M, redO, P, B, shift, c->cg,
                                   c->cgpart, c->scal));
    if ((s = cr_check_launch(c, "cg_apply")) != CR_OK) return s;
    cudaError_t e = cudaMemcpyAsync(out, c->cg + 6 * (size_t)P, (size_t)P * 16,
                                    cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess && u_out)
        e = cudaMemcpyAsync(u_out, c->u_tmp, (size_t)B * 2 * sizeof(R), cudaMemcpyDeviceToDevice,
                            c->stream);
    return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "sr_sv copy: %s", cudaGetErrorString(e));
}

extern "C" cr_status sr_sv(cr_ctx* ctx, const int8_t* spins, const void* tanh_theta, int B,
                           const double* v, double shift, void* u_out, double* out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(B >= 1 && B <= ctx->max_walkers, "sr_sv: B=%d outside [1, %d]", B,
                 ctx->max_walkers);
    CR_CHECK_ARG(spins && tanh_theta && v && out, "sr_sv: null array");
    CR_CHECK_ARG(shift >= 0.0, "sr_sv: shift must be >= 0");
    return ctx->prec == CR_FP64 ? sv_t<double>(ctx, spins, tanh_theta, B, v, shift, u_out, out)
                                : sv_t<float>(ctx, spins, tanh_theta, B, v, shift, u_out, out);
}

template <typename R>
static cr_status smatrix_t(cr_ctx* c, const int8_t* spins, const void* T, int B, double shift,
                           double* S_out) {
    double* redO = c->red + 2 * (c->P + 2 + c->M);
    cr_status s = oreduce(c, false, spins, T, nullptr, B, redO, nullptr);
    if (s != CR_OK) return s;
    if ((s = build_s<R>(c, spins, T, B, redO, shift)) != CR_OK) return s;
    cudaError_t e = cudaMemcpyAsync(S_out, c->S, (size_t)c->P * c->P * 16,
                                    cudaMemcpyDeviceToDevice, c->stream);
    return e == cudaSuccess ? CR_OK : cr_fail(c, CR_ECUDA, "sr_smatrix copy: %s", cudaGetErrorString(e));
}

extern "C" cr_status sr_smatrix(cr_ctx* ctx, const int8_t* spins, const void* tanh_theta, int B,
                                double shift, double* S_out) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(ctx->flags & CR_CTX_EXPLICIT_S,
                 "sr_smatrix: needs a context created with CR_CTX_EXPLICIT_S");
    CR_CHECK_ARG(B >= 1 && B <= ctx->max_walkers, "sr_smatrix: B=%d outside [1, %d]", B,
                 ctx->max_walkers);
    CR_CHECK_ARG(spins && tanh_theta && S_out, "sr_smatrix: null array");
    CR_CHECK_ARG(shift >= 0.0, "sr_smatrix: shift must be >= 0");
    return ctx->prec == CR_FP64 ? smatrix_t<double>(ctx, spins, tanh_theta, B, shift, S_out)
                                : smatrix_t<float>(ctx, spins, tanh_theta, B, shift, S_out);
}

// ------------------------------------------------------ backward of log psi

template <typename R>
__global__ void to_params_kernel(const double* __restrict__ red_, int P, cpx<R>* __restrict__ out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P) out[k] = ccast<R>(((const cpx<double>*)red_)[k]);
}

extern "C" cr_status logpsi_backward(cr_ctx* ctx, const cr_state* st, const int8_t* spins,
                                     const void* tanh_theta, int B, const void* grad_logpsi,
                                     void* grad_params) {
    if (!ctx) return CR_EINVAL;
    CR_CHECK_ARG(st && grad_params, "logpsi_backward: null state or output");
    CR_CHECK_ARG(B >= 0 && B <= ctx->max_walkers, "logpsi_backward: B=%d outside [0, %d]", B,
                 ctx->max_walkers);
    const int P = ctx->P;
    if (B == 0) {
        cudaError_t e = cudaMemsetAsync(grad_params, 0, (size_t)P * 2 * rsize(ctx), ctx->stream);
        return e == cudaSuccess ? CR_OK : cr_fail(ctx, CR_ECUDA, "memset: %s", cudaGetErrorString(e));
    }
    CR_CHECK_ARG(spins && tanh_theta && grad_logpsi, "logpsi_backward: null array");
    double* red = ctx->red;
    cr_status s = oreduce(ctx, true, spins, tanh_theta, grad_logpsi, B, red, nullptr);
    if (s != CR_OK) return s;
    if (ctx->prec == CR_FP64)
        CR_LAUNCH(ctx, CR_K_OTHER, to_params_kernel<double><<<(P + 255) / 256, 256, 0, ctx->stream>>>(red, P,
                                                                          (cpx<double>*)grad_params));
    else
        CR_LAUNCH(ctx, CR_K_OTHER, to_params_kernel<float><<<(P + 255) / 256, 256, 0, ctx->stream>>>(red, P,
                                                                         (cpx<float>*)grad_params));
    return cr_check_launch(ctx, "to_params");
}

// ------------------------------------- VJP of log psi without allocation
//
// For callers that cannot allocate device memory themselves: code running
// inside a framework whose caching allocator owns the device's memory
// budget, plugins and services given a fixed footprint, or callers that
// must not trigger the device-wide synchronisation cudaFree implies.  The
// reduction scratch of logpsi_backward is a fixed array in the library's
// own device image instead of context workspace.

// 4 MiB of float64: partial rows [chunks][P + 2 + M] complex128 followed by
// the reduced row [P + 2] complex128.  Every GPU that loads the library
// holds it until the process exits.
#define CR_NOALLOC_SCRATCH_DOUBLES (512 * 1024)
static __device__ __align__(256) double g_noalloc_scratch[CR_NOALLOC_SCRATCH_DOUBLES];

#define CR_NOALLOC_MAX_DEVICES 64
static double* g_noalloc_ptr[CR_NOALLOC_MAX_DEVICES];

static void noalloc_err(char* buf, int len, const char* msg) {
    if (buf && len > 0) {
        strncpy(buf, msg, (size_t)len - 1);
        buf[len - 1] = '\0';
    }
}

template <typename R>
static cudaError_t noalloc_backward_t(int N, int M, const int8_t* spins, const void* T, int B,
                                      const void* g, void* grad, int nch, double* scratch,
                                      cudaStream_t st) {
    const int P = N + M + N * M;
    const int chunk = (B + nch - 1) / nch;
    const int jpt = (M + 127) / 128;
    const bool dbl = sizeof(R) == 8;
    double* red = scratch + (size_t)nch * (P + 2 + M) * 2;
#define LAUNCH(JPT, IT)                                                                    \
    oreduce_kernel<R, JPT, IT, true, true><<<dim3(nch, (N + IT - 1) / IT), 128, 0, st>>>(  \
        spins, (const cpx<R>*)T, (const cpx<R>*)g, B, N, M, P, chunk, scratch, nullptr)
    if (jpt == 1) {
        if (dbl) LAUNCH(1, 8); else LAUNCH(1, 16);
    } else if (jpt == 2) {
        if (dbl) LAUNCH(2, 4); else LAUNCH(2, 8);
    } else {
        if (dbl) LAUNCH(4, 2); else LAUNCH(4, 4);
    }
#undef LAUNCH
    combine_kernel<double><<<(P + 2 + 255) / 256, 256, 0, st>>>(scratch, nch, P + 2, P + 2 + M,
                                                                 red, nullptr);
    to_params_kernel<R><<<(P + 255) / 256, 256, 0, st>>>(red, P, (cpx<R>*)grad);
    return cudaGetLastError();
}

extern "C" cr_status logpsi_backward_noalloc(int N, int M, cr_prec prec, const int8_t* spins,
                                             const void* tanh_theta, int B,
                                             const void* grad_logpsi, void* grad_params,
                                             void* stream, char* errbuf, int errbuf_len) {
    if (N < 2 || N > 1024 || M < 1 || M > 512 || B < 0) {
        noalloc_err(errbuf, errbuf_len, "logpsi_backward_noalloc: need 2 <= N <= 1024, "
                                        "1 <= M <= 512, B >= 0");
        return CR_EINVAL;
    }
    if (prec != CR_FP64 && prec != CR_FP32 && prec != CR_MIXED) {
        noalloc_err(errbuf, errbuf_len, "logpsi_backward_noalloc: unknown precision");
        return CR_EINVAL;
    }
    const long long P = (long long)N + M + (long long)N * M;
    const long long row = 2 * (P + 2 + M), tail = 2 * (P + 2);
    long long nch = (CR_NOALLOC_SCRATCH_DOUBLES - tail) / row;
    if (nch < 1) {
        noalloc_err(errbuf, errbuf_len, "logpsi_backward_noalloc: N + M + N*M too large for "
                                        "the 4 MiB scratch (limit about 131000 parameters)");
        return CR_EINVAL;
    }
    if (!grad_params || (B > 0 && (!spins || !tanh_theta || !grad_logpsi))) {
        noalloc_err(errbuf, errbuf_len, "logpsi_backward_noalloc: null array");
        return CR_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rs = prec == CR_FP64 ? 8 : 4;
    if (B == 0) {
        cudaError_t e = cudaMemsetAsync(grad_params, 0, (size_t)P * 2 * rs, st);
        if (e != cudaSuccess) {
            noalloc_err(errbuf, errbuf_len, cudaGetErrorString(e));
            return CR_ECUDA;
        }
        return CR_OK;
    }
    // once per device, with that device current: the device address of the
    // scratch array (in host code its name is only a host-side stand-in)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= CR_NOALLOC_MAX_DEVICES) {
        noalloc_err(errbuf, errbuf_len, "logpsi_backward_noalloc: no usable current device");
        return CR_ECUDA;
    }
    double* scratch = __atomic_load_n(&g_noalloc_ptr[dev], __ATOMIC_ACQUIRE);
    if (!scratch) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            noalloc_err(errbuf, errbuf_len, "logpsi_backward_noalloc: cudaGetSymbolAddress failed");
            return CR_ECUDA;
        }
        scratch = (double*)p;
        __atomic_store_n(&g_noalloc_ptr[dev], scratch, __ATOMIC_RELEASE);
    }
    if (nch > 64) nch = 64;
    if (nch > B) nch = B;
    // a launch error still pending from earlier, unrelated work on this thread
    // is not this call's failure: clear it before the launches below
    (void)cudaGetLastError();
    e = prec == CR_FP64 ? noalloc_backward_t<double>(N, M, spins, tanh_theta, B, grad_logpsi,
                                                     grad_params, (int)nch, scratch, st)
                        : noalloc_backward_t<float>(N, M, spins, tanh_theta, B, grad_logpsi,
                                                    grad_params, (int)nch, scratch, st);
    if (e != cudaSuccess) {
        noalloc_err(errbuf, errbuf_len, cudaGetErrorString(e));
        return CR_ECUDA;
    }
    return CR_OK;
}
