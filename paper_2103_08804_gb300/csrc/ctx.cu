// Context lifetime, workspace and status handling.
#include <stdarg.h>
#include <stdlib.h>

#include <vector>

#include "common.cuh"

cr_status tc_prepare(cr_ctx* c);
cr_status target_prepare(cr_ctx* c);
cr_status sym_prepare(cr_ctx* c);
void sgram_geometry(const cr_ctx* c, int* R2, int* nkc_max, size_t* plane_bytes, int* npl);
std::vector<int2> sgram_tiles(int P);

cr_status cr_fail(cr_ctx* c, cr_status s, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

bool cr_kt_begin(cr_ctx* c, int kid) {
    if (kid < 0 || c->kt.kid != kid || c->kt.count >= c->kt.cap) return false;
    // launches being captured into a graph are not timed: an event record
    // would only become a graph node, never a timestamp of this launch
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return false;
    cudaEventRecord(c->kt.ev[2 * c->kt.count], c->stream);
    return true;
}

void cr_kt_end(cr_ctx* c) {
    cudaEventRecord(c->kt.ev[2 * c->kt.count + 1], c->stream);
    ++c->kt.count;
}

static void kt_free(cr_ctx* c) {
    if (c->kt.ev) {
        for (int i = 0; i < 2 * c->kt.cap; ++i) cudaEventDestroy(c->kt.ev[i]);
        free(c->kt.ev);
    }
    c->kt.ev = nullptr;
    c->kt.cap = c->kt.count = 0;
    c->kt.kid = -1;
}

extern "C" long long cr_n_launches(const cr_ctx* c) { return c ? c->n_launches : -1; }

extern "C" cr_status cr_time_kernel(cr_ctx* c, int kid, int cap) {
    if (!c) return CR_EINVAL;
    kt_free(c);
    if (kid < 0) return CR_OK;
    if (cap < 1) return cr_fail(c, CR_EINVAL, "cr_time_kernel: capacity < 1");
    c->kt.ev = (cudaEvent_t*)calloc(2 * (size_t)cap, sizeof(cudaEvent_t));
    if (!c->kt.ev) return CR_ENOMEM;
    for (int i = 0; i < 2 * cap; ++i)
        if (cudaEventCreate(&c->kt.ev[i]) != cudaSuccess) {
            c->kt.cap = i / 2;
            kt_free(c);
            return cr_fail(c, CR_ECUDA, "cr_time_kernel: event creation failed");
        }
    c->kt.cap = cap;
    c->kt.count = 0;
    c->kt.kid = kid;
    return CR_OK;
}

extern "C" int cr_kernel_times(cr_ctx* c, float* ms, int cap) {
    if (!c || !ms) return -1;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return -1;
    int n = c->kt.count < cap ? c->kt.count : cap;
    for (int i = 0; i < n; ++i)
        if (cudaEventElapsedTime(&ms[i], c->kt.ev[2 * i], c->kt.ev[2 * i + 1]) != cudaSuccess)
            return -1;
    return n;
}

cr_status cr_check_launch(cr_ctx* c, const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cr_fail(c, CR_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return CR_OK;
}

// Periodic nearest-neighbour bonds: (r, r + x-hat) for all r, then
// (r, r + y-hat) for all r when Ly > 1 (Sec. V: nearest neighbours, PBC).
static std::vector<int2> make_bonds(int Lx, int Ly) {
    std::vector<int2> b;
    for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) b.push_back(make_int2(x + Lx * y, (x + 1) % Lx + Lx * y));
    if (Ly > 1)
        for (int y = 0; y < Ly; ++y)
            for (int x = 0; x < Lx; ++x) b.push_back(make_int2(x + Lx * y, x + Lx * ((y + 1) % Ly)));
    return b;
}

static cudaError_t alloc(void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(p, bytes);
}

extern "C" cr_status cr_create(cr_ctx** out, const cr_lattice* lat, int M, int max_walkers,
                               cr_prec prec, int flags, void* stream) {
    if (!out || !lat) return CR_EINVAL;
    *out = nullptr;
    if (lat->Lx < 3 || lat->Ly < 1 || (lat->Ly != 1 && lat->Ly < 3)) return CR_EINVAL;
    if (M < 1 || M > 512 || max_walkers < 1) return CR_EINVAL;
    if (prec != CR_FP64 && prec != CR_FP32 && prec != CR_MIXED) return CR_EINVAL;
    cr_ctx* c = (cr_ctx*)calloc(1, sizeof(cr_ctx));
    if (!c) return CR_ENOMEM;
    c->Lx = lat->Lx;
    c->Ly = lat->Ly;
    c->N = lat->Lx * lat->Ly;
    c->M = M;
    // hidden units padded to 32 lanes x a power-of-two run per lane
    int kpl = 1;
    while (32 * kpl < M) kpl *= 2;
    c->Mp = 32 * kpl;
    c->Nb = lat->Ly == 1 ? c->N : 2 * c->N;
    c->P = c->N + M + c->N * M;
    c->J = lat->J;
    c->prec = prec;
    c->max_walkers = max_walkers;
    c->flags = flags;
    c->stream = (cudaStream_t)stream;
    c->kt.kid = -1;
    // walker chunks of the reductions: enough CTAs to fill the GPU, each chunk
    // at least 128 walkers; partial rows cost (P + 2 + M) x 16 bytes each
    c->n_chunks = (max_walkers + 127) / 128;
    if (c->n_chunks > 128) c->n_chunks = 128;
    c->max_chunks = c->n_chunks;
    if (c->N > 1024 || c->N % 2) {
        free(c);
        return CR_EINVAL;
    }
    const size_t rs = rsize(c), cs = 2 * rs;
    const size_t P = c->P, Nb = c->Nb, Mp = c->Mp, B = max_walkers;
    cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes)                                 \
    if (e == cudaSuccess) e = alloc((void**)&(ptr), (bytes))
    ALLOC(c->d_status, sizeof(int));
    ALLOC(c->d_bonds, Nb * sizeof(int2));
    for (int s = 0; s < 2; ++s) {
        ALLOC(c->tab[s].D, Nb * Mp * cs);
        ALLOC(c->tab[s].Ch, Nb * Mp * cs);
        ALLOC(c->tab[s].Sh, Nb * Mp * cs);
        ALLOC(c->tab[s].ChT, Nb * Mp * cs);
        ALLOC(c->tab[s].ShT, Nb * Mp * cs);
        ALLOC(c->tab[s].ea, Nb * 2 * cs);
    }
    ALLOC(c->theta_tmp, B * M * cs);
    ALLOC(c->lp_tmp, 2 * B * cs);
    ALLOC(c->u_tmp, B * cs);
    ALLOC(c->partial, (size_t)c->n_chunks * (P + 2 + M) * 16);
    ALLOC(c->red, 3 * (P + 2 + M) * 16);
    ALLOC(c->F, P * 16);
    ALLOC(c->cg, 5 * P * 16);
    ALLOC(c->p_lo, P * cs);
    size_t ncgpart = (P + 31) / 32 + 2 * ((P + 255) / 256);
    if (ncgpart < chol_cgpart_len()) ncgpart = chol_cgpart_len();
    ALLOC(c->cgpart, ncgpart * sizeof(double));
    ALLOC(c->scal, 64 * sizeof(double));
    std::vector<int2> gt;
    if (flags & CR_CTX_EXPLICIT_S) {
        ALLOC(c->S, P * P * 16);
        if (prec == CR_MIXED) {
            int R2, nkc, npl;
            size_t pb;
            sgram_geometry(c, &R2, &nkc, &pb, &npl);
            gt = sgram_tiles(c->P);
            c->n_gtiles = (int)gt.size();
            ALLOC(c->Xt, npl * pb);
            ALLOC(c->gtiles, gt.size() * sizeof(int2));
        } else {
            ALLOC(c->O_tmp, B * P * cs);
        }
        if (chol_blocked(c)) ALLOC(c->Lf, chol_factor_bytes(c));
    }
    int dev = 0;
    c->n_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess)
        cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, dev);
    std::vector<int2> ot;
    if (prec == CR_MIXED) {
        size_t xb, pb;
        ored_sizes(c, &xb, &pb, &ot);
        ALLOC(c->ored_x, xb);
        ALLOC(c->ored_part, pb);
        ALLOC(c->ored_tiles, ot.size() * sizeof(int2));
    }
    c->fcg = e == cudaSuccess && fcg_supported(c) ? 1 : 0;
    if (c->fcg) {
        size_t a1, b2, v2p, part;
        fcg_sizes(c, &a1, &b2, &v2p, &part);
        c->fcg_v2plane = v2p;
        ALLOC(c->fcg_a1, a1);
        ALLOC(c->fcg_b2, b2);
        ALLOC(c->fcg_v2, 3 * v2p);
        ALLOC(c->fcg_vab, (size_t)(c->N + M) * 8);
        ALLOC(c->fcg_part, part);
        ALLOC(c->fcg_psc, (size_t)c->n_sm * 8 * sizeof(double));
        ALLOC(c->fcg_bar, 4 * sizeof(unsigned));
        // padding entries of the V planes (sites past N, columns past 2M) stay zero
        if (e == cudaSuccess) e = cudaMemset(c->fcg_v2, 0, 3 * v2p);
    }
#undef ALLOC
    if (e != cudaSuccess) {
        cr_destroy(c);
        return e == cudaErrorMemoryAllocation ? CR_ENOMEM : CR_ECUDA;
    }
    if (cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cr_destroy(c);
        return CR_ECUDA;
    }
    std::vector<int2> bonds = make_bonds(c->Lx, c->Ly);
    e = cudaMemcpy(c->d_bonds, bonds.data(), Nb * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !gt.empty())
        e = cudaMemcpy(c->gtiles, gt.data(), gt.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !ot.empty()) {
        e = cudaMemcpy(c->ored_tiles, ot.data(), ot.size() * sizeof(int2), cudaMemcpyHostToDevice);
        c->ored = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->scal, 0, 64 * sizeof(double));
    if (e != cudaSuccess || tc_prepare(c) != CR_OK || target_prepare(c) != CR_OK || sym_prepare(c) != CR_OK ||
        (c->fcg && fcg_prepare(c) != CR_OK)) {
        cr_destroy(c);
        return CR_ECUDA;
    }
    *out = c;
    return CR_OK;
}

extern "C" cr_status cr_destroy(cr_ctx* c) {
    if (!c) return CR_EINVAL;
    kt_free(c);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    void* ptrs[] = {c->d_status, c->d_bonds, c->theta_tmp, c->lp_tmp, c->u_tmp, c->partial,
                    c->red, c->F, c->cg, c->p_lo, c->cgpart, c->scal, c->S, c->O_tmp, c->kry,
                    c->Lf, c->Xt, c->gtiles, c->fcg_a1, c->fcg_b2, c->fcg_v2, c->fcg_vab,
                    c->fcg_part, c->fcg_psc, c->fcg_bar, c->gram_x, c->gram_part,
                    c->gram_tiles, c->lp_work, c->ored_x, c->ored_part, c->ored_tiles};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int s = 0; s < 2; ++s) {
        void* t[] = {c->tab[s].D, c->tab[s].Ch, c->tab[s].Sh, c->tab[s].ChT, c->tab[s].ShT,
                     c->tab[s].ea};
        for (void* p : t)
            if (p) cudaFree(p);
    }
    free(c);
    return CR_OK;
}

cr_status cr_grow(cr_ctx* c, void** p, size_t* cap, size_t need, const char* who) {
    if (*cap >= need) return CR_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        (void)cudaGetLastError();
        *p = nullptr;
        return cr_fail(c, CR_ENOMEM, "%s: cannot allocate %zu bytes of scratch", who, need);
    }
    *cap = need;
    return CR_OK;
}

extern "C" cr_status cr_set_stream(cr_ctx* c, void* stream) {
    if (!c) return CR_EINVAL;
    c->stream = (cudaStream_t)stream;
    return CR_OK;
}

extern "C" cr_status cr_set_chunks(cr_ctx* c, int n_chunks) {
    if (!c) return CR_EINVAL;
    if (n_chunks < 1 || n_chunks > c->max_chunks)
        return cr_fail(c, CR_EINVAL, "n_chunks %d outside [1, %d]", n_chunks, c->max_chunks);
    c->n_chunks = n_chunks;
    return CR_OK;
}

extern "C" int cr_max_chunks(const cr_ctx* c) { return c ? c->max_chunks : -1; }

extern "C" const char* cr_last_error(const cr_ctx* c) { return c ? c->err : "null context"; }

extern "C" cr_status cr_sync_status(cr_ctx* c) {
    if (!c) return CR_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cr_fail(c, CR_ECUDA, "stream sync: %s", cudaGetErrorString(e));
    int st = 0;
    e = cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return cr_fail(c, CR_ECUDA, "status read: %s", cudaGetErrorString(e));
    if (st) cr_fail(c, (cr_status)st, "device status %d", st);
    return (cr_status)st;
}

extern "C" int cr_fused_cg(const cr_ctx* c) { return c ? c->fcg : -1; }

extern "C" cr_status cr_set_fcg_ctas(cr_ctx* c, int n_ctas) {
    if (!c) return CR_EINVAL;
    if (!c->fcg) return cr_fail(c, CR_EINVAL, "cr_set_fcg_ctas: no fused CG in this context");
    if (n_ctas < 0 || n_ctas > c->n_sm)
        return cr_fail(c, CR_EINVAL, "cr_set_fcg_ctas: %d outside [0, %d]", n_ctas, c->n_sm);
    c->fcg_ctas = n_ctas;
    return CR_OK;
}

// One natural-gradient iteration of a sequence, on its context's stream.
static cr_status seq_iteration(const cr_seq_iter* q) {
    cr_ctx* c = q->ctx;
    cr_state st = {q->params, 0, 0.0, 0.0};
    cr_status s = mc_sweep(c, &st, q->spins, q->theta, q->B, q->n_sweeps, q->rng, q->logpsi,
                           q->tanh_theta, nullptr);
    if (s == CR_OK) s = cheb_local_target(c, &q->target, q->spins, q->logpsi, q->B, q->R, nullptr);
    if (s == CR_OK) s = sr_step(c, q->params, q->spins, q->tanh_theta, q->R, q->B, &q->opts, q->stats);
    if (s == CR_OK) s = rbm_logpsi(c, &st, q->spins, q->B, q->theta, q->logpsi);
    return s;
}

extern "C" cr_status cr_batch_run(const cr_seq_iter* seqs, int n, int n_iter, void* stream) {
    if (!seqs || n < 1 || n_iter < 0) return CR_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!seqs[i].ctx) return CR_EINVAL;
        for (int j = 0; j < i; ++j)
            if (seqs[j].ctx == seqs[i].ctx)
                return cr_fail(seqs[i].ctx, CR_EINVAL, "cr_batch_run: a context appears twice");
    }
    cudaStream_t main = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        cr_ctx* c = seqs[i].ctx;
        if (cudaEventRecord(c->ev_fork, main) != cudaSuccess ||
            cudaStreamWaitEvent(c->stream, c->ev_fork, 0) != cudaSuccess)
            return cr_fail(c, CR_ECUDA, "cr_batch_run: fork");
    }
    cr_status st = CR_OK;
    for (int it = 0; it < n_iter && st == CR_OK; ++it)
        for (int i = 0; i < n && st == CR_OK; ++i) st = seq_iteration(&seqs[i]);
    // join every stream, also after a failure, so that the caller's stream
    // orders after whatever was enqueued
    for (int i = 0; i < n; ++i) {
        cr_ctx* c = seqs[i].ctx;
        if (cudaEventRecord(c->ev_join, c->stream) != cudaSuccess ||
            cudaStreamWaitEvent(main, c->ev_join, 0) != cudaSuccess)
            return cr_fail(c, CR_ECUDA, "cr_batch_run: join");
    }
    return st;
}
extern "C" int cr_n_sites(const cr_ctx* c) { return c ? c->N : -1; }
extern "C" int cr_n_hidden(const cr_ctx* c) { return c ? c->M : -1; }
extern "C" int cr_n_params(const cr_ctx* c) { return c ? c->P : -1; }
extern "C" int cr_n_bonds(const cr_ctx* c) { return c ? c->Nb : -1; }
