// C ABI of the slab factor+solve library: validation, device memory plan,
// orchestration of the phases of Algorithms 3 and 4, and FP64 iterative
// refinement on top of the (FP32 or FP64) factor.
#include <algorithm>
#include <atomic>
#include <thread>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cstdio>
#include <limits>

#include "slab_internal.cuh"

slab_status slab_cuda_check(slab_handle* h, cudaError_t e, const char* file, int line) {
    static const bool trace = std::getenv("SLAB_CUDA_TRACE") != nullptr;
    if (trace) std::fprintf(stderr, "slab: %s at %s:%d\n", cudaGetErrorString(e), file, line);
    if (h && h->err == SLAB_OK) h->err = SLAB_ECUDA;
    return SLAB_ECUDA;
}

namespace {

slab_status dalloc(slab_handle* h, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return SLAB_OK;
    if (h->arena) {
        SlabArena* A = h->arena;
        const size_t off = (A->off + 255) & ~(size_t)255;
        if (A->base && off + bytes > A->cap) return SLAB_ENOMEM;
        *p = A->base + off;                            // sizing pass: an offset, never dereferenced
        A->off = off + bytes;
        h->dev_bytes += (int64_t)bytes;
        return SLAB_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SLAB_ENOMEM;
    }
    h->dev_bytes += (int64_t)bytes;
    return SLAB_OK;
}

void dfree(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

void free_workspace(slab_handle* h) {
    dfree(h->wYv); dfree(h->wGtb); dfree(h->wXs); dfree(h->wFi); dfree(h->wX); dfree(h->wZ);
    dfree(h->t3y); dfree(h->t3G); dfree(h->t3x); dfree(h->t3Fi); dfree(h->t3xI);
    dfree(h->wVp);
    dfree(h->wVtk);
    dfree(h->wPart);
    void* tk0 = h->wTickets; dfree(tk0); h->wTickets = nullptr;
    void* r = h->wR; dfree(r); h->wR = nullptr;
    void* q = h->wNrm; dfree(q); h->wNrm = nullptr;
    void* rp = h->red_part; dfree(rp); h->red_part = nullptr;
    void* tk = h->red_tickets; dfree(tk); h->red_tickets = nullptr;
    h->red_cap = h->ticket_cap = 0;
    h->kcap = 0;
    h->rcap = 0;
}

#define TRY(x)                            \
    do {                                  \
        slab_status _s = (x);             \
        if (_s != SLAB_OK) return _s;     \
    } while (0)

// Stage-1 solve phases by dimension
template <typename T>
slab_status up_gather(slab_handle* h, const double* F, double fscale, int r0, int K) {
    return h->dim == 3 ? tree3d_up_gather<T>(h, F, fscale, r0, K) : tree_up_gather<T>(h, F, fscale, r0, K);
}
template <typename T>
slab_status down_scatter(slab_handle* h, double* U, int accumulate, int r0, int K) {
    return h->dim == 3 ? tree3d_down_scatter<T>(h, U, accumulate, r0, K) : tree_down_scatter<T>(h, U, accumulate, r0, K);
}
template <typename T>
slab_status export_x(slab_handle* h, double* out, double scale, int r0, int K) {
    return h->dim == 3 ? tree3d_export<T>(h, out, scale, r0, K) : export_ftilde_part<T>(h, out, scale, r0, K);
}
template <typename T>
slab_status import_x(slab_handle* h, const double* in, int r0, int K) {
    return h->dim == 3 ? tree3d_import<T>(h, in, r0, K) : import_utilde_part<T>(h, in, r0, K);
}

// Solve workspace for up to kc right-hand sides per pass and k total (residual buffer).
slab_status ensure_workspace(slab_handle* h, int k) {
    const int kc = k < tree_kmax() ? k : tree_kmax();
    const TreeDims& d = h->td;
    static_assert(sizeof(double) == 8, "");
    if (h->kcap < kc) {
        const int64_t nodes = (int64_t)d.NS * (d.s + 1);
        dfree(h->wYv); dfree(h->wGtb); dfree(h->wXs); dfree(h->wFi); dfree(h->wX); dfree(h->wZ);
        dfree(h->wX2); dfree(h->wZ2);
        dfree(h->t3y); dfree(h->t3G); dfree(h->t3x); dfree(h->t3Fi); dfree(h->t3xI);
        h->kcap = 0;
        if (h->dim == 3) {
            const int64_t nn = tree3d_nodes(h->t3plan);
            const int64_t Mp = tree3d_mpad(h->t3plan);
            TRY(dalloc(h, &h->t3y, nn * kc * Mp * h->rsz));
            TRY(dalloc(h, &h->t3x, nn * kc * Mp * h->rsz));
            TRY(dalloc(h, &h->t3G, nn * kc * 2 * Mp * h->rsz));
            TRY(dalloc(h, &h->t3Fi, (int64_t)d.NS * 2 * kc * d.s_pad * h->rsz));
            TRY(dalloc(h, &h->t3xI, tree3d_xI_elems(h->t3plan) * kc * h->rsz));
        } else {
            TRY(dalloc(h, &h->wYv, nodes * d.m * kc * h->rsz));
            TRY(dalloc(h, &h->wGtb, nodes * 2 * d.m * kc * h->rsz));
            TRY(dalloc(h, &h->wXs, nodes * d.m * kc * h->rsz));
            TRY(dalloc(h, &h->wFi, (int64_t)d.NS * 2 * d.s_pad * kc * h->rsz));
        }
        TRY(dalloc(h, &h->wX, (int64_t)d.NI * d.s_pad * kc * h->rsz));
        TRY(dalloc(h, &h->wZ, (int64_t)d.NI * d.s_pad * kc * h->rsz));
        if (h->prec2 != h->prec) {
            TRY(dalloc(h, &h->wX2, (int64_t)d.NI * d.s_pad * kc * h->rsz2));
            TRY(dalloc(h, &h->wZ2, (int64_t)d.NI * d.s_pad * kc * h->rsz2));
        }
        h->kcap = kc;
    }
    if (!h->wVtk && h->dim == 2) {
        const size_t e = tree_down_ws_elems(d.s, d.m, d.NS);
        TRY(dalloc(h, &h->wVp, (e ? e : 1) * h->rsz));
        const size_t nt = tree_down_tickets(d.s, d.NS);
        TRY(dalloc(h, &h->wVtk, nt * sizeof(unsigned)));
        if (!sizing_pass(h)) SLAB_CK(h, cudaMemsetAsync(h->wVtk, 0, nt * sizeof(unsigned), h->stream));
    }
    if (!h->wPart) {
        TRY(dalloc(h, &h->wPart, splitk_part_bytes(d.s_pad)));
        void* tk = nullptr;
        TRY(dalloc(h, &tk, (size_t)(d.s_pad / SLAB_TILE) * sizeof(unsigned)));
        h->wTickets = (unsigned*)tk;
        if (!sizing_pass(h))
            SLAB_CK(h, cudaMemsetAsync(h->wTickets, 0, (size_t)(d.s_pad / SLAB_TILE) * sizeof(unsigned), h->stream));
    }
    return SLAB_OK;
}

// FP64 residual buffer and norms for k right-hand sides.
slab_status ensure_resid(slab_handle* h, int k) {
    const int64_t N = h->td.N;
    if (h->rcap < k) {
        void* r = h->wR; dfree(r); h->wR = nullptr;
        void* q = h->wNrm; dfree(q); h->wNrm = nullptr;
        h->rcap = 0;
        TRY(dalloc(h, &r, (size_t)k * N * sizeof(double)));
        h->wR = (double*)r;
        TRY(dalloc(h, &q, (size_t)2 * k * sizeof(double)));
        h->wNrm = (double*)q;
        h->rcap = k;
    }
    return SLAB_OK;
}

// Mixed mode: the interface sweep runs in the Stage-2 scalar on wX2 / wZ2, which this view
// swaps in for wX / wZ for its lifetime.
struct Stage2Vectors {
    slab_handle* h;
    explicit Stage2Vectors(slab_handle* hh) : h(hh) { swap(); }
    ~Stage2Vectors() { swap(); }
    void swap() {
        void* t = h->wX; h->wX = h->wX2; h->wX2 = t;
        t = h->wZ; h->wZ = h->wZ2; h->wZ2 = t;
    }
};

// Algorithm 2 on the interface vectors wX (Stage-1 scalar), in the Stage-2 scalar.
slab_status interface_sweep(slab_handle* h, int K) {
    if (h->prec2 == h->prec)
        return h->prec == SLAB_PREC_FP64 ? sweep_solve<double>(h, K) : sweep_solve<float>(h, K);
    const int64_t n = (int64_t)h->td.NI * h->kcap * h->td.s_pad;
    TRY(widen_to_double(h, (const float*)h->wX, (double*)h->wX2, n));
    {
        Stage2Vectors v(h);
        TRY(sweep_solve<double>(h, K));
    }
    return narrow_to_float(h, (const double*)h->wX2, (float*)h->wX, n);
}

template <typename T>
slab_status solve_pass(slab_handle* h, const double* F, double fscale, double* U, int accumulate, int k) {
    const int kc = h->kcap;
    for (int r0 = 0; r0 < k; r0 += kc) {
        const int K = (k - r0) < kc ? (k - r0) : kc;
        if (h->dim == 3) {
            TRY(tree3d_up_gather<T>(h, F, fscale, r0, K));
            TRY(interface_sweep(h, K));
            TRY(tree3d_down_scatter<T>(h, U, accumulate, r0, K));
        } else {
            TRY(tree_up_gather<T>(h, F, fscale, r0, K));
            TRY(interface_sweep(h, K));
            TRY(tree_down_scatter<T>(h, U, accumulate, r0, K));
        }
    }
    return SLAB_OK;
}

slab_status pass(slab_handle* h, const double* F, double fscale, double* U, int accumulate, int k) {
    return h->prec == SLAB_PREC_FP64 ? solve_pass<double>(h, F, fscale, U, accumulate, k)
                                     : solve_pass<float>(h, F, fscale, U, accumulate, k);
}

}  // namespace

slab_status slab_dalloc(slab_handle* h, void** p, size_t bytes) { return dalloc(h, p, bytes); }

slab_status solve_prepare(slab_handle* h, int k) {
    TRY(ensure_workspace(h, k));
    TRY(ensure_resid(h, k));
    return ensure_red(h, k);
}

slab_status reset_scratch(slab_handle* h) {
    if (h->wVtk && h->dim == 2)
        SLAB_CK(h, cudaMemsetAsync(h->wVtk, 0, tree_down_tickets(h->td.s, h->td.NS) * sizeof(unsigned), h->stream));
    if (h->wTickets)
        SLAB_CK(h, cudaMemsetAsync(h->wTickets, 0, (size_t)(h->td.s_pad / SLAB_TILE) * sizeof(unsigned), h->stream));
    if (h->red_tickets) SLAB_CK(h, cudaMemsetAsync(h->red_tickets, 0, h->ticket_cap * sizeof(unsigned), h->stream));
    return SLAB_OK;
}

slab_status solve_fixed(slab_handle* h, const double* f, double* u, int k, int steps, double* nrm) {
    const double h2 = 1.0 / ((double)h->n * (double)h->n);
    TRY(pass(h, f, h2, u, 0, k));
    for (int it = 0; it < steps; ++it) {
        TRY(launch_residual(h, u, f, h->wR, k, nullptr, nullptr));
        TRY(pass(h, h->wR, h2, u, 1, k));
    }
    SLAB_CK(h, cudaMemsetAsync(nrm, 0, 2 * (size_t)k * sizeof(double), h->stream));
    return launch_residual(h, u, f, h->wR, k, nrm, nrm + k);
}

bool slab_debug() {
    static const bool on = std::getenv("SLAB_DEBUG") != nullptr;
    return on;
}

unsigned slab_debug_status(slab_handle* h, const char* where, int a, int b) {
    cudaStreamSynchronize(h->stream);
    unsigned st = 0;
    cudaMemcpy(&st, h->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (st) std::fprintf(stderr, "slab: status 0x%x after %s (%d, %d)\n", st, where, a, b);
    return st;
}

namespace {

slab_status sync_status(slab_handle* h) {
    SLAB_CK(h, cudaStreamSynchronize(h->stream));
    unsigned st = 0;
    SLAB_CK(h, cudaMemcpy(&st, h->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (st & SLAB_DEV_TIMEOUT) {
        if (h->err == SLAB_OK) h->err = SLAB_ETIMEOUT;
        return SLAB_ETIMEOUT;
    }
    if (st & SLAB_DEV_NOTSPD) {
        if (h->err == SLAB_OK) h->err = SLAB_ESINGULAR;
        return SLAB_ESINGULAR;
    }
    return SLAB_OK;
}

// Stage 1 and the assembly of T (into h->Tb / h->To in the Stage-1 scalar)
template <typename T>
slab_status stage1_impl(slab_handle* h) {
    if (h->dim == 3) {
        h->stage1_dense = 1;
        const slab_status st = tree3d_factor<T>(h);
        h->stage1_dense = 0;
        return st;
    }
    TRY(tree_factor<T>(h));
    return assemble_T<T>(h);
}

template <typename T>
slab_status factor_impl(slab_handle* h) {
    if (h->prec2 == h->prec) {
        TRY(stage1_impl<T>(h));
        h->fp64tc_now = h->fp64tc;
        const slab_status st = sweep_factor<T>(h);
        h->fp64tc_now = 0;
        return st;
    }
    // mixed mode: assemble T in the Stage-1 scalar, widen it, eliminate in the Stage-2 scalar
    void* Tb2 = h->Tb;
    void* To2 = h->To;
    void* Tl2 = h->Tl;
    h->Tb = h->Tb1;
    h->To = h->To1;
    h->Tl = h->Tl1;
    const slab_status st = stage1_impl<T>(h);
    h->Tb = Tb2;
    h->To = To2;
    h->Tl = Tl2;
    TRY(st);
    const int64_t blk = (int64_t)h->td.s_pad * h->td.s_pad;
    TRY(widen_to_double(h, (const float*)h->Tb1, (double*)h->Tb, h->td.NI * blk));
    TRY(widen_to_double(h, (const float*)h->To1, (double*)h->To, (h->td.NI - 1) * blk));
    if (h->Tl) TRY(widen_to_double(h, (const float*)h->Tl1, (double*)h->Tl, (h->td.NI - 1) * blk));
    h->fp64tc_now = h->fp64tc;
    const slab_status st2 = sweep_factor<double>(h);
    h->fp64tc_now = 0;
    return st2;
}

}  // namespace

slab_status factor_status(slab_handle* h) { return sync_status(h); }

namespace {

struct ProfRecord {
    std::vector<cudaEvent_t> pool;     // event pairs, reused
    std::vector<int> cls;              // class of each recorded pair
    size_t used = 0;
    cudaEvent_t pending = nullptr;
};

}  // namespace

void prof_begin(slab_handle* h, int cls) {
    if (!h) return;
    cls = prof_class(h, cls);
    h->launches[cls] += 1;
    if (!h->prof_on || !h->prof) return;
    ProfRecord* R = (ProfRecord*)h->prof;
    if (R->pool.size() < 2 * (R->used + 1)) {
        for (int i = 0; i < 64; ++i) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return;
            R->pool.push_back(e);
        }
    }
    cudaEventRecord(R->pool[2 * R->used], h->stream);
    R->cls.resize(R->used + 1);
    R->cls[R->used] = cls;
}

void prof_end(slab_handle* h, int cls) {
    (void)cls;
    if (!h || !h->prof_on || !h->prof) return;
    ProfRecord* R = (ProfRecord*)h->prof;
    if (R->cls.size() != R->used + 1) return;
    cudaEventRecord(R->pool[2 * R->used + 1], h->stream);
    R->used += 1;
}

static void prof_free(slab_handle* h) {
    if (!h->prof) return;
    ProfRecord* R = (ProfRecord*)h->prof;
    for (auto e : R->pool) cudaEventDestroy(e);
    delete R;
    h->prof = nullptr;
}

extern "C" {

slab_status slab_profile(slab_handle* h, int enable) {
    if (!h) return SLAB_EINVAL;
    if (enable && !h->prof) h->prof = new (std::nothrow) ProfRecord();
    h->prof_on = enable && h->prof;
    return SLAB_OK;
}

slab_status slab_profile_read(slab_handle* h, double* ms, int64_t* launches, int n) {
    if (!h || n < 0 || n > SLAB_KERNEL_CLASSES) return SLAB_EINVAL;
    SLAB_CK(h, cudaStreamSynchronize(h->stream));
    for (int c = 0; c < n; ++c) {
        if (ms) ms[c] = 0.0;
        if (launches) launches[c] = h->launches[c];
    }
    for (int c = 0; c < SLAB_KERNEL_CLASSES; ++c) h->launches[c] = 0;
    if (h->prof) {
        ProfRecord* R = (ProfRecord*)h->prof;
        for (size_t i = 0; i < R->used; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, R->pool[2 * i], R->pool[2 * i + 1]) == cudaSuccess && ms && R->cls[i] < n)
                ms[R->cls[i]] += t;
        }
        R->used = 0;
        R->cls.clear();
    }
    return SLAB_OK;
}


void slab_default_opts(slab_opts* o) {
    if (!o) return;
    o->factor_prec = SLAB_PREC_FP32;
    o->pivot = 0;
    o->rtol = 1e-10;
    o->max_refine = 30;
    o->krylov = 0;
    o->stream = nullptr;
    o->profile = 0;
    o->stage2 = SLAB_STAGE2_AUTO;
    o->interface_prec = -1;
}

const char* slab_strerror(slab_status s) {
    switch (s) {
        case SLAB_OK: return "ok";
        case SLAB_EINVAL: return "invalid argument";
        case SLAB_ENOMEM: return "device allocation failed";
        case SLAB_ESINGULAR: return "non-positive or zero pivot in a factorisation";
        case SLAB_ENOCONV: return "iterative refinement did not reach the tolerance";
        case SLAB_ETIMEOUT: return "bounded device wait gave up";
        case SLAB_ECUDA: return "CUDA runtime error";
        case SLAB_EUNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

void slab_destroy(slab_handle* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    const cudaStream_t own = h->own_stream ? h->stream : nullptr;
    if (h->arena) {                                    // buffers belong to the arena's owner
        if (h->t3plan) tree3d_plan_free(h->t3plan);
        if (own) cudaStreamDestroy(own);
        prof_free(h);
        delete h;
        return;
    }
    free_workspace(h);
    dfree(h->wX2); dfree(h->wZ2);
    {
        void* q = h->kV; dfree(q); q = h->kZ; dfree(q); q = h->kS; dfree(q);
    }
    void* p;
    p = h->AX; dfree(p); p = h->AY; dfree(p); p = h->DG; dfree(p); p = h->kappa; dfree(p);
    dfree(h->tLinv); dfree(h->tZtb); dfree(h->tRtb); dfree(h->tZI); dfree(h->tRI);
    dfree(h->tWtb); dfree(h->tWI); dfree(h->ToT); dfree(h->dscratch);
    p = h->AXT; dfree(p); p = h->AYT; dfree(p);
    dfree(h->tLinvT); dfree(h->tZtbT); dfree(h->tWtbT); dfree(h->tZIT); dfree(h->tWIT); dfree(h->tRIc);
    dfree(h->Tl); dfree(h->Tl1); dfree(h->SinvT); dfree(h->WT); dfree(h->TlT); dfree(h->gjw); dfree(h->ozw); dfree(h->w16); dfree(h->pnl);
    p = h->AZ; dfree(p);
    dfree(h->t3Lin); dfree(h->t3LT); dfree(h->t3Ztb); dfree(h->t3ZtbT); dfree(h->t3ZIT); dfree(h->t3ZI);
    dfree(h->t3Rtb); dfree(h->t3RI); dfree(h->t3W);
    if (h->t3plan) tree3d_plan_free(h->t3plan);
    if (own) cudaStreamDestroy(own);
    dfree(h->Tb); dfree(h->To); dfree(h->Fct); dfree(h->Linv); dfree(h->Y);
    dfree(h->crD); dfree(h->crE); dfree(h->crW); dfree(h->crLT); dfree(h->Tb1); dfree(h->To1);
    dfree(h->crPt); dfree(h->crP); dfree(h->crQt); dfree(h->crQ);
    p = h->dstatus; dfree(p);
    prof_free(h);
    delete h;
}

}  // extern "C"

namespace {

// Elimination order of an FP32 Stage 2 when the caller leaves it open.  Both orders run one
// tall Cholesky per eliminated block, whose s_pad / 64 panel steps are latency-bound (about
// 35 us each: two small launches and a thin update, measured on GB300), while the products run
// at a few hundred TFLOP/s.  The sweep eliminates N_I blocks one after another with about
// 2.7 s_pad^3 flops each; the odd-even order eliminates a whole level per batch (so only the
// levels count towards the panel latency) but does about 3 s_pad^3 per eliminated block plus
// 5 s_pad^3 per block with a right neighbour.  Pick the smaller modelled time.
bool oddeven_is_faster(int NI, int s_pad) {
    const double panel_s = 35e-6, rate = 3e14;
    const double P = s_pad / 64.0, s3 = (double)s_pad * s_pad * s_pad;
    int levels = 0, nb = 0, nc = 0;
    for (int step = 1; step < NI; step *= 2) {
        const int nrem = (NI - 1) / step + 1;
        if (nrem < 2) break;
        ++levels;
        nb += nrem / 2;
        nc += (nrem - 1) / 2;
    }
    const double t_sweep = NI * P * panel_s + NI * 2.7 * s3 / rate;
    const double t_oe = (levels + 1) * P * panel_s + (nb * 3.0 + nc * 5.0 + 1.0) * s3 / rate;
    return t_oe < t_sweep;
}

}  // namespace

// slab_factor in three steps, so that a batch can allocate everything first and record only
// launches in a CUDA graph: factor_create validates and allocates (no kernel runs), factor_launch
// enqueues the factor on h->stream (no allocation, no host synchronisation), factor_finish waits,
// reads the device status word and frees the factor-only buffers.
slab_status factor_create(const slab_grid* grid, const slab_coeffs* co, int b, const slab_opts* opts,
                          slab_handle** out, SlabArena* arena) {
    if (!grid || !co || !out) return SLAB_EINVAL;
    *out = nullptr;
    slab_opts o;
    if (opts) o = *opts;
    else slab_default_opts(&o);
    const int n = grid->n;
    if (grid->dim != 2 && grid->dim != 3) return SLAB_EINVAL;
    if (b < 2 || n < 4 || n % b != 0 || n / b < 2) return SLAB_EINVAL;
    if (co->kind < SLAB_POISSON || co->kind > SLAB_CONVECTION) return SLAB_EINVAL;
    if ((co->kind == SLAB_DIFFUSION || co->kind == SLAB_CONVECTION) && !co->kappa) return SLAB_EINVAL;
    if (co->kind == SLAB_CONVECTION && !co->beta) return SLAB_EINVAL;
    if (co->kind == SLAB_HELMHOLTZ && !co->c) return SLAB_EINVAL;
    if (o.factor_prec < SLAB_PREC_FP64 || o.factor_prec > SLAB_PREC_TF32) return SLAB_EINVAL;
    const int want_tf32 = o.factor_prec == SLAB_PREC_TF32 || o.interface_prec == SLAB_PREC_TF32;
    const int want_fp64tc = o.interface_prec == SLAB_PREC_FP64_TC;
    if (want_fp64tc) o.interface_prec = SLAB_PREC_FP64;
    if (o.factor_prec == SLAB_PREC_TF32) o.factor_prec = SLAB_PREC_FP32;
    if (o.interface_prec == SLAB_PREC_TF32) o.interface_prec = SLAB_PREC_FP32;
    if (o.stage2 < SLAB_STAGE2_AUTO || o.stage2 > SLAB_STAGE2_ODDEVEN) return SLAB_EINVAL;
    if (o.krylov < 0 || o.krylov > 200) return SLAB_EINVAL;
    if (o.pivot < 0 || o.pivot > 1) return SLAB_EINVAL;
    int prec2 = o.interface_prec;
    if (prec2 == -1) prec2 = (co->kind == SLAB_HELMHOLTZ) ? SLAB_PREC_FP64 : o.factor_prec;
    if (prec2 != SLAB_PREC_FP32 && prec2 != SLAB_PREC_FP64) return SLAB_EINVAL;
    if (o.factor_prec == SLAB_PREC_FP64 && prec2 == SLAB_PREC_FP32) return SLAB_EINVAL;
    if (grid->dim == 2 && b - 1 > SLAB_MAXM) return SLAB_EUNSUPPORTED;
    const bool general = co->kind == SLAB_HELMHOLTZ || co->kind == SLAB_CONVECTION;   // LU, not Cholesky
    const bool nonsym = co->kind == SLAB_CONVECTION;
    if (grid->dim == 3 && general) return SLAB_EUNSUPPORTED;
    if (o.stage2 == SLAB_STAGE2_ODDEVEN && general) return SLAB_EUNSUPPORTED;

    slab_handle* h = new (std::nothrow) slab_handle();
    if (!h) return SLAB_ENOMEM;
    std::memset(h, 0, sizeof(*h));
    h->arena = arena;
    h->dim = grid->dim; h->n = n; h->b = b; h->kind = co->kind; h->omega = co->omega;
    h->beta = nonsym ? co->beta : nullptr;
    h->prec = o.factor_prec;
    h->rsz = h->prec == SLAB_PREC_FP64 ? 8 : 4;
    h->tf32 = want_tf32;
    h->fp64tc = want_fp64tc;
    h->prec2 = prec2;
    h->rsz2 = h->prec2 == SLAB_PREC_FP64 ? 8 : 4;
    h->stream = (cudaStream_t)o.stream;
    h->rtol = o.rtol;
    h->max_refine = o.max_refine;
    h->krylov = o.krylov;
    h->pivot_local = o.pivot == 1;
    if (o.profile) slab_profile(h, 1);
    TreeDims& d = h->td;
    d.s = n - 1;
    d.si = grid->dim == 3 ? d.s * d.s : d.s;
    d.N = (int64_t)d.si * d.s;
    d.s_pad = (d.si + SLAB_TILE - 1) / SLAB_TILE * SLAB_TILE;
    d.m = b - 1;
    d.H = tree_height_count(d.s);
    d.NS = n / b;
    d.NI = d.NS - 1;
    d.b = b;
    d.n = n;
    h->nt = d.s_pad / SLAB_TILE;

    slab_status st = SLAB_OK;
    const size_t nodes2 = (size_t)(n + 1) * (n + 1) * (grid->dim == 3 ? (size_t)(n + 1) : 1);
    const size_t R = h->rsz;
    const size_t R2 = h->rsz2;
    const int64_t tn = (int64_t)d.NS * (d.s + 1);
    const int64_t blk = (int64_t)d.s_pad * d.s_pad;
    void* p;
#define ALLOC(field, bytes)                             \
    do {                                                \
        st = dalloc(h, &p, (bytes));                    \
        if (st) { slab_destroy(h); return st; }         \
        field = decltype(field)(p);                     \
    } while (0)
    ALLOC(h->AX, nodes2 * sizeof(double));
    ALLOC(h->AY, nodes2 * sizeof(double));
    ALLOC(h->DG, nodes2 * sizeof(double));
    if (co->kind == SLAB_DIFFUSION || nonsym) ALLOC(h->kappa, nodes2 * sizeof(double));
    if (nonsym) {
        ALLOC(h->AXT, nodes2 * sizeof(double));
        ALLOC(h->AYT, nodes2 * sizeof(double));
    }
    if (grid->dim == 3) {
        ALLOC(h->AZ, nodes2 * sizeof(double));
        h->t3plan = tree3d_plan(d.s, d.m, d.NS);
        const int64_t nn = tree3d_nodes(h->t3plan);
        const int64_t Mp = tree3d_mpad(h->t3plan);
        ALLOC(h->t3Lin, nn * Mp * Mp * R);
        ALLOC(h->t3LT, nn * Mp * Mp * R);
        ALLOC(h->t3Ztb, nn * 2 * Mp * Mp * R);
        ALLOC(h->t3ZtbT, nn * 2 * Mp * Mp * R);
        ALLOC(h->t3ZIT, tree3d_zit_elems(h->t3plan) * R);
        ALLOC(h->t3ZI, tree3d_zit_elems(h->t3plan) * R);
        ALLOC(h->t3Rtb, nn * 4 * Mp * Mp * R);
        ALLOC(h->t3RI, (int64_t)d.NS * d.H * 4 * Mp * d.s_pad * R);
        ALLOC(h->t3W, tree3d_work_elems(h->t3plan) * R);
    } else {
        ALLOC(h->tLinv, tn * d.m * d.m * R);
        ALLOC(h->tZtb, tn * 2 * d.m * d.m * R);
        ALLOC(h->tRtb, tn * 4 * d.m * d.m * R);
        ALLOC(h->tZI, (int64_t)d.NS * d.H * 2 * d.m * d.s_pad * R);
        ALLOC(h->tRI, (int64_t)d.NS * d.H * 4 * d.m * d.s_pad * R);
        if (nonsym) {
            ALLOC(h->tLinvT, tn * d.m * d.m * R);
            ALLOC(h->tZtbT, tn * 2 * d.m * d.m * R);
            ALLOC(h->tWtbT, tn * 2 * d.m * d.m * R);
            ALLOC(h->tZIT, (int64_t)d.NS * d.H * 2 * d.m * d.s_pad * R);
            ALLOC(h->tWIT, (int64_t)d.NS * d.H * 2 * d.m * d.s_pad * R);
            ALLOC(h->tRIc, (int64_t)d.NS * d.H * 4 * d.m * d.s_pad * R);
        }
    }
    ALLOC(h->Tb, d.NI * blk * R2);
    ALLOC(h->To, (d.NI - 1) * blk * R2);
    if (nonsym) ALLOC(h->Tl, (d.NI - 1) * blk * R2);
    if (h->prec2 != h->prec) {
        ALLOC(h->Tb1, d.NI * blk * R);
        ALLOC(h->To1, (d.NI - 1) * blk * R);
        if (nonsym) ALLOC(h->Tl1, (d.NI - 1) * blk * R);
    }
    h->stage2 = o.stage2 == SLAB_STAGE2_ODDEVEN ||
                (o.stage2 == SLAB_STAGE2_AUTO && !general && d.NI >= 4 &&
                 h->prec2 == SLAB_PREC_FP32 && oddeven_is_faster(d.NI, d.s_pad));
    if (h->stage2) {
        ALLOC(h->crD, d.NI * blk * R2);
        ALLOC(h->crE, (d.NI > 1 ? d.NI - 1 : 1) * blk * R2);
        ALLOC(h->crW, (int64_t)cr_max_batch(d.NI) * 2 * blk * R2);
        ALLOC(h->crLT, d.NI * blk * R2);
        ALLOC(h->crPt, d.NI * blk * R2);
        ALLOC(h->crP, d.NI * blk * R2);
        ALLOC(h->crQt, d.NI * blk * R2);
        ALLOC(h->crQ, d.NI * blk * R2);
    } else if (general) {
        ALLOC(h->Fct, 5 * blk * R2);                    // augmented system [S | T | I] over [T | T]
        ALLOC(h->gjw, gj_work_bytes(d.s_pad, R2));
    } else {
        ALLOC(h->Fct, d.NI * 3 * blk * R2);
    }
    if (general) {
        ALLOC(h->tWtb, tn * 2 * d.m * d.m * R);
        ALLOC(h->tWI, (int64_t)d.NS * d.H * 2 * d.m * d.s_pad * R);
        if (!nonsym) ALLOC(h->ToT, (d.NI - 1) * blk * R2);     // T_{q+1,q} = T_{q,q+1}^T
    }
    if (nonsym) {                                               // the A^T sweep
        ALLOC(h->SinvT, d.NI * blk * R2);
        ALLOC(h->WT, (d.NI - 1) * blk * R2);
        ALLOC(h->TlT, (d.NI - 1) * blk * R2);
    }
    ALLOC(h->dscratch, 256);
    if (h->fp64tc) ALLOC(h->ozw, ozaki_work_bytes(2 * (int64_t)d.s_pad + 128, 3 * (int64_t)d.s_pad, 64));
    if (!h->tf32 && !general &&
        (h->prec2 == SLAB_PREC_FP32 || (h->dim == 3 && h->prec == SLAB_PREC_FP32))) {
        // largest FP16 three-product of the factor: the batched Stage-2 Schur products (s_pad^3)
        h->w16_bytes = f16x3_work_bytes(d.s_pad, d.s_pad, d.s_pad, h->stage2 ? cr_max_batch(d.NI) : 1, false);
        ALLOC(h->w16, h->w16_bytes);
    }
    ALLOC(h->Linv, d.NI * blk * R2);
    if (!h->stage2) ALLOC(h->Y, (d.NI - 1) * blk * R2);
    ALLOC(h->dstatus, sizeof(unsigned));
    {
        // panel inverses of the tall Cholesky: two 64 x 64 blocks per matrix of its largest batch
        int pb = h->stage2 ? cr_max_batch(d.NI) : 1;
        if (grid->dim == 3) pb = std::max(pb, d.NS * tree_nodes_at(d.s, 0));
        h->pnl_bytes = 2 * (size_t)std::min(pb, 65535) * SLAB_TILE * SLAB_TILE * std::max(R, R2);
        ALLOC(h->pnl, h->pnl_bytes);
    }
#undef ALLOC
    *out = h;
    return SLAB_OK;
}

// Enqueue the factor of a created handle for the coefficients co (read during the launches).
slab_status factor_launch(slab_handle* h, const double* kappa, const double* c) {
    const TreeDims& d = h->td;
    const size_t R = h->rsz;
    const size_t nodes2 = (size_t)(h->n + 1) * (h->n + 1) * (h->dim == 3 ? (size_t)(h->n + 1) : 1);
    SLAB_CK(h, cudaMemsetAsync(h->dstatus, 0, sizeof(unsigned), h->stream));
    if (h->tZI) SLAB_CK(h, cudaMemsetAsync(h->tZI, 0, (size_t)d.NS * d.H * 2 * d.m * d.s_pad * R, h->stream));
    if (h->tRI) SLAB_CK(h, cudaMemsetAsync(h->tRI, 0, (size_t)d.NS * d.H * 4 * d.m * d.s_pad * R, h->stream));
    if (h->tWI) SLAB_CK(h, cudaMemsetAsync(h->tWI, 0, (size_t)d.NS * d.H * 2 * d.m * d.s_pad * R, h->stream));
    if (h->tZIT) SLAB_CK(h, cudaMemsetAsync(h->tZIT, 0, (size_t)d.NS * d.H * 2 * d.m * d.s_pad * R, h->stream));
    if (h->tWIT) SLAB_CK(h, cudaMemsetAsync(h->tWIT, 0, (size_t)d.NS * d.H * 2 * d.m * d.s_pad * R, h->stream));
    if (h->tRIc) SLAB_CK(h, cudaMemsetAsync(h->tRIc, 0, (size_t)d.NS * d.H * 4 * d.m * d.s_pad * R, h->stream));
    if (h->kappa && kappa != h->kappa)
        SLAB_CK(h, cudaMemcpyAsync(h->kappa, kappa, nodes2 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    slab_status st = launch_coefficients(h, kappa, c);
    h->tf32_now = h->tf32;
    if (!st) st = h->prec == SLAB_PREC_FP64 ? factor_impl<double>(h) : factor_impl<float>(h);
    h->tf32_now = 0;
    return st;
}

static void free_factor_only(slab_handle* h) {
    dfree(h->Tb1);                                     // mixed-mode assembly buffers
    dfree(h->To1);
    dfree(h->Tl1);
    h->Tb1 = h->To1 = h->Tl1 = nullptr;
    dfree(h->tRIc);                                    // condensed couplings (nonsymmetric kind)
    dfree(h->w16);                                     // factor-only product work
    h->w16 = nullptr;
    h->w16_bytes = 0;
    dfree(h->pnl);
    h->pnl = nullptr;
    h->pnl_bytes = 0;
    dfree(h->t3Rtb);                                   // 3-D factor-only arrays
    dfree(h->t3RI);
    dfree(h->t3W);
}

extern "C" {

slab_status slab_factor(const slab_grid* grid, const slab_coeffs* co, int b, const slab_opts* opts,
                        slab_handle** out) {
    if (!out) return SLAB_EINVAL;
    *out = nullptr;
    slab_handle* h = nullptr;
    slab_status st = factor_create(grid, co, b, opts, &h, nullptr);
    if (st) return st;
    st = factor_launch(h, co->kappa, co->c);
    if (!st) st = sync_status(h);
    h->beta = nullptr;                                 // the caller's field is read during the call only
    if (st) {
        slab_destroy(h);
        return st;
    }
    free_factor_only(h);
    *out = h;
    return SLAB_OK;
}

slab_status slab_apply_residual(slab_handle* h, const double* u, const double* f, double* r, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!u || !f || !r) return SLAB_EINVAL;
    return launch_residual(h, u, f, r, k, nullptr, nullptr);
}

slab_status slab_boundary_lift(slab_handle* h, const double* g, const double* f, double* f_out, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!g || !f_out) return SLAB_EINVAL;
    if (h->kind == SLAB_CONVECTION) return SLAB_EUNSUPPORTED;
    return launch_boundary_lift(h, g, f, f_out, k);
}

slab_status slab_apply_transpose(slab_handle* h, const double* x, double* y, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!x || !y) return SLAB_EINVAL;
    h->transposed = h->kind == SLAB_CONVECTION;
    const slab_status st = launch_apply(h, x, y, k);
    h->transposed = 0;
    return st;
}

slab_status slab_apply(slab_handle* h, const double* x, double* y, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!x || !y) return SLAB_EINVAL;
    return launch_apply(h, x, y, k);
}

namespace {

// Krylov arrays for k right-hand sides: basis V [m+1][k][N], directions Z [m][k][N], and the
// small device arrays (H columns [m+1][k], combination coefficients [m][k], dot partials, norms).
slab_status ensure_krylov(slab_handle* h, int k) {
    if (h->kcapk >= k) return SLAB_OK;
    const int m = h->krylov;
    const int64_t N = h->td.N;
    void* p = h->kV; dfree(p); p = h->kZ; dfree(p); p = h->kS; dfree(p);
    h->kV = h->kZ = h->kS = nullptr;
    h->kcapk = 0;
    TRY(dalloc(h, &p, (size_t)(m + 1) * k * N * sizeof(double)));
    h->kV = (double*)p;
    TRY(dalloc(h, &p, (size_t)m * k * N * sizeof(double)));
    h->kZ = (double*)p;
    TRY(dalloc(h, &p, ((size_t)(2 * m + 1) * k + vec_dot_part_elems(k) + 2 * (size_t)k) * sizeof(double)));
    h->kS = (double*)p;
    h->kcapk = k;
    return SLAB_OK;
}

// Refinement by restarted right-preconditioned GMRES(m) in FP64, one Krylov space per
// right-hand side: the preconditioner is one solve pass with the factor, u0 = M^{-1} f, and each
// restart starts from the true FP64 residual.  The preconditioned directions are kept (flexible
// form), since the FP32 solve is linear only up to rounding.  max_refine bounds the number of
// preconditioner applications after the first.
slab_status gmres_solve(slab_handle* h, const double* f, double* u, int k, double* relres_out, int* iters_out) {
    const int m = h->krylov;
    const int64_t N = h->td.N;
    const int64_t kN = (int64_t)k * N;
    const double h2 = 1.0 / ((double)h->n * (double)h->n);
    TRY(ensure_workspace(h, k));
    TRY(ensure_krylov(h, k));
    double* V = h->kV;
    double* Z = h->kZ;
    double* Hd = h->kS;                                  // [m+1][k]
    double* Cd = Hd + (size_t)(m + 1) * k;               // [m][k]
    double* part = Cd + (size_t)m * k;
    double* nrm = part + vec_dot_part_elems(k);          // [2][k]: ||r||^2, ||f||^2
    TRY(pass(h, f, h2, u, 0, k));
    std::vector<double> hb((size_t)(m + 1) * k), nh(2 * (size_t)k), fn(k);
    std::vector<double> R((size_t)k * m * m), cs((size_t)k * m), sn((size_t)k * m), g((size_t)k * (m + 1));
    std::vector<double> coef((size_t)m * k);
    int it = 0;
    slab_status result = SLAB_OK;
    for (;;) {
        SLAB_CK(h, cudaMemsetAsync(nrm, 0, 2 * k * sizeof(double), h->stream));
        TRY(launch_residual(h, u, f, V, k, nrm, nrm + k));
        SLAB_CK(h, cudaMemcpyAsync(nh.data(), nrm, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        SLAB_CK(h, cudaStreamSynchronize(h->stream));
        double worst = 0.0;
        bool finite = true;
        for (int q = 0; q < k; ++q) {
            fn[q] = nh[k + q] > 0 ? std::sqrt(nh[k + q]) : 1.0;
            double rr;
            if (!std::isfinite(nh[q])) {
                rr = std::numeric_limits<double>::quiet_NaN();
                finite = false;
            } else {
                rr = nh[q] > 0 ? std::sqrt(nh[q]) / fn[q] : 0.0;
            }
            if (relres_out) relres_out[q] = rr;
            if (!(rr <= worst)) worst = rr;
        }
        if (!finite) { result = SLAB_ENOCONV; break; }
        if (worst <= h->rtol) break;
        if (it >= h->max_refine) { result = SLAB_ENOCONV; break; }
        TRY(vec_scale(h, V, nrm, N, k));                 // v_0 = r / ||r||
        for (int q = 0; q < k; ++q) {
            std::fill(g.begin() + (size_t)q * (m + 1), g.begin() + (size_t)(q + 1) * (m + 1), 0.0);
            g[(size_t)q * (m + 1)] = std::sqrt(nh[q] > 0 ? nh[q] : 0.0);
        }
        int jdone = 0;
        for (int j = 0; j < m; ++j) {
            double* Vj = V + (int64_t)j * kN;
            double* Vn = V + (int64_t)(j + 1) * kN;
            double* Zj = Z + (int64_t)j * kN;
            TRY(pass(h, Vj, h2, Zj, 0, k));                // z_j = M^{-1} v_j
            ++it;
            TRY(launch_apply(h, Zj, Vn, k));               // w = A z_j
            for (int i = 0; i <= j; ++i) {                 // modified Gram-Schmidt
                TRY(vec_dot(h, Vn, V + (int64_t)i * kN, N, k, part, Hd + (size_t)i * k));
                TRY(vec_axpy(h, Vn, V + (int64_t)i * kN, Hd + (size_t)i * k, -1.0, N, k));
            }
            TRY(vec_dot(h, Vn, Vn, N, k, part, Hd + (size_t)(j + 1) * k));
            TRY(vec_scale(h, Vn, Hd + (size_t)(j + 1) * k, N, k));
            SLAB_CK(h, cudaMemcpyAsync(hb.data(), Hd, (size_t)(j + 2) * k * sizeof(double), cudaMemcpyDeviceToHost,
                                       h->stream));
            SLAB_CK(h, cudaStreamSynchronize(h->stream));
            double est = 0.0;
            for (int q = 0; q < k; ++q) {
                double* col = R.data() + ((size_t)q * m + j) * m;          // column j of R (rows 0..j)
                double* c = cs.data() + (size_t)q * m;
                double* s = sn.data() + (size_t)q * m;
                double* gq = g.data() + (size_t)q * (m + 1);
                std::vector<double> r(j + 2);
                for (int i = 0; i <= j; ++i) r[i] = hb[(size_t)i * k + q];
                const double hn = hb[(size_t)(j + 1) * k + q];
                r[j + 1] = hn > 0 ? std::sqrt(hn) : 0.0;
                for (int i = 0; i < j; ++i) {
                    const double t = c[i] * r[i] + s[i] * r[i + 1];
                    r[i + 1] = -s[i] * r[i] + c[i] * r[i + 1];
                    r[i] = t;
                }
                const double d = std::hypot(r[j], r[j + 1]);
                c[j] = d > 0 ? r[j] / d : 1.0;
                s[j] = d > 0 ? r[j + 1] / d : 0.0;
                r[j] = d;
                gq[j + 1] = -s[j] * gq[j];
                gq[j] = c[j] * gq[j];
                for (int i = 0; i <= j; ++i) col[i] = r[i];
                est = std::max(est, std::fabs(gq[j + 1]) / fn[q]);
            }
            jdone = j + 1;
            if (!(est > 0.5 * h->rtol) || it >= h->max_refine) break;
        }
        for (int q = 0; q < k; ++q) {                    // y = R^{-1} g, back substitution
            const double* gq = g.data() + (size_t)q * (m + 1);
            std::vector<double> y(jdone, 0.0);
            for (int i = jdone - 1; i >= 0; --i) {
                double acc = gq[i];
                for (int l = i + 1; l < jdone; ++l) acc -= R[((size_t)q * m + l) * m + i] * y[l];
                const double di = R[((size_t)q * m + i) * m + i];
                y[i] = di != 0.0 ? acc / di : 0.0;
            }
            for (int i = 0; i < jdone; ++i) coef[(size_t)i * k + q] = y[i];
        }
        SLAB_CK(h, cudaMemcpyAsync(Cd, coef.data(), (size_t)jdone * k * sizeof(double), cudaMemcpyHostToDevice,
                                   h->stream));
        TRY(vec_combine(h, u, Z, kN, Cd, jdone, k, N));   // u += Z y
    }
    if (iters_out) *iters_out = it;
    return result;
}

}  // namespace

slab_status slab_solve(slab_handle* h, const double* f, double* u, int k, double* relres_out, int* iters_out) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) {
        if (iters_out) *iters_out = 0;
        return SLAB_OK;
    }
    if (!f || !u) return SLAB_EINVAL;
    if (h->krylov > 0 && h->max_refine > 0) {
        TRY(ensure_resid(h, k));
        return gmres_solve(h, f, u, k, relres_out, iters_out);
    }
    TRY(ensure_workspace(h, k));
    const double h2 = 1.0 / ((double)h->n * (double)h->n);
    TRY(pass(h, f, h2, u, 0, k));
    int it = 0;
    slab_status result = SLAB_OK;
    if (h->max_refine > 0 || relres_out) {
        TRY(ensure_resid(h, k));
        std::vector<double> nrm(2 * (size_t)k);
        double prev = -1.0;
        int stall = 0;
        bool have_f = false;                        // ||f||^2 is computed with the first residual only
        for (;;) {
            SLAB_CK(h, cudaMemsetAsync(h->wNrm, 0, (have_f ? 1 : 2) * k * sizeof(double), h->stream));
            TRY(launch_residual(h, u, f, h->wR, k, h->wNrm, have_f ? nullptr : h->wNrm + k));
            SLAB_CK(h, cudaMemcpyAsync(nrm.data(), h->wNrm, (have_f ? 1 : 2) * k * sizeof(double),
                                       cudaMemcpyDeviceToHost, h->stream));
            have_f = true;
            SLAB_CK(h, cudaStreamSynchronize(h->stream));
            double worst = 0.0;
            bool finite = true;
            for (int q = 0; q < k; ++q) {
                double rr;
                if (!std::isfinite(nrm[q])) {           // the iterate holds Inf / NaN
                    rr = std::numeric_limits<double>::quiet_NaN();
                    finite = false;
                } else {
                    rr = nrm[q] > 0 ? std::sqrt(nrm[q] / (nrm[k + q] > 0 ? nrm[k + q] : 1.0)) : 0.0;
                }
                if (relres_out) relres_out[q] = rr;
                if (!(rr <= worst)) worst = rr;
            }
            if (!finite) {
                result = SLAB_ENOCONV;
                break;
            }
            if (worst <= h->rtol) break;
            // stagnation: two consecutive steps without halving the worst residual
            stall = (prev > 0.0 && worst > 0.5 * prev) ? stall + 1 : 0;
            prev = worst;
            if (it >= h->max_refine || stall >= 2) {
                result = h->max_refine > 0 ? SLAB_ENOCONV : SLAB_OK;
                break;
            }
            TRY(pass(h, h->wR, h2, u, 1, k));
            ++it;
        }
    }
    if (iters_out) *iters_out = it;
    return result;
}

slab_status slab_adjoint(slab_handle* h, const double* dLdu, const double* u, double* lambda, double* dLdkappa,
                         int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!dLdu || !lambda) return SLAB_EINVAL;
    if (dLdkappa && ((h->kind != SLAB_DIFFUSION && h->kind != SLAB_CONVECTION) || !u)) return SLAB_EINVAL;
    if (dLdkappa && h->dim != 2) return SLAB_EUNSUPPORTED;
    // A^T lambda = dL/du with the same factors: the symmetric kinds' solve is slab_solve's; the
    // nonsymmetric kind runs every phase transposed (tree passes, sweep, residual)
    h->transposed = h->kind == SLAB_CONVECTION;
    slab_status st = slab_solve(h, dLdu, lambda, k, nullptr, nullptr);
    h->transposed = 0;
    if (st != SLAB_OK && st != SLAB_ENOCONV) return st;
    if (dLdkappa) TRY(launch_kappa_gradient(h, u, lambda, dLdkappa, k));
    return st;
}

slab_status slab_reduced_rhs(slab_handle* h, const double* f, double* ftilde, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!f || !ftilde) return SLAB_EINVAL;
    TRY(ensure_workspace(h, k));
    const double h2 = 1.0 / ((double)h->n * (double)h->n);
    for (int r0 = 0; r0 < k; r0 += h->kcap) {
        const int K = (k - r0) < h->kcap ? (k - r0) : h->kcap;
        if (h->prec == SLAB_PREC_FP64) {
            TRY(up_gather<double>(h, f, h2, r0, K));
            TRY(export_x<double>(h, ftilde, 1.0 / h2, r0, K));
        } else {
            TRY(up_gather<float>(h, f, h2, r0, K));
            TRY(export_x<float>(h, ftilde, 1.0 / h2, r0, K));
        }
    }
    return SLAB_OK;
}

slab_status slab_interface_solve(slab_handle* h, const double* ftilde, double* utilde, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!ftilde || !utilde) return SLAB_EINVAL;
    TRY(ensure_workspace(h, k));
    const double h2 = 1.0 / ((double)h->n * (double)h->n);
    for (int r0 = 0; r0 < k; r0 += h->kcap) {
        const int K = (k - r0) < h->kcap ? (k - r0) : h->kcap;
        if (h->prec2 != h->prec) {
            Stage2Vectors v(h);
            TRY(import_x<double>(h, ftilde, r0, K));
            TRY(sweep_solve<double>(h, K));
            TRY(export_x<double>(h, utilde, h2, r0, K));
        } else if (h->prec == SLAB_PREC_FP64) {
            TRY(import_x<double>(h, ftilde, r0, K));
            TRY(sweep_solve<double>(h, K));
            TRY(export_x<double>(h, utilde, h2, r0, K));
        } else {
            TRY(import_x<float>(h, ftilde, r0, K));
            TRY(sweep_solve<float>(h, K));
            TRY(export_x<float>(h, utilde, h2, r0, K));
        }
    }
    return SLAB_OK;
}

slab_status slab_interior_solve(slab_handle* h, const double* f, const double* utilde, double* u, int k) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!f || !utilde || !u) return SLAB_EINVAL;
    TRY(ensure_workspace(h, k));
    const double h2 = 1.0 / ((double)h->n * (double)h->n);
    for (int r0 = 0; r0 < k; r0 += h->kcap) {
        const int K = (k - r0) < h->kcap ? (k - r0) : h->kcap;
        if (h->prec == SLAB_PREC_FP64) {
            TRY(up_gather<double>(h, f, h2, r0, K));
            TRY(import_x<double>(h, utilde, r0, K));
            TRY(down_scatter<double>(h, u, 0, r0, K));
        } else {
            TRY(up_gather<float>(h, f, h2, r0, K));
            TRY(import_x<float>(h, utilde, r0, K));
            TRY(down_scatter<float>(h, u, 0, r0, K));
        }
    }
    return SLAB_OK;
}

slab_status slab_apply_T(slab_handle* h, const double* X, double* Y, int k, double* work) {
    if (!h || k < 0) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!X || !Y || !work) return SLAB_EINVAL;
    // u_I = X and u_J = -A_JJ^-1 A_JI X (interior solve with zero load), then (A u)_I = T X
    const int64_t N = h->td.N;
    double* f0 = work;
    double* u = work + (int64_t)k * N;
    SLAB_CK(h, cudaMemsetAsync(f0, 0, (size_t)k * N * sizeof(double), h->stream));
    TRY(slab_interior_solve(h, f0, X, u, k));
    TRY(launch_apply(h, u, f0, k));
    return launch_gather_interface(h, f0, Y, k);
}

slab_status slab_get_T_block(slab_handle* h, int which, int q, double* out) {
    if (!h || !out || which < 0 || which > 2) return SLAB_EINVAL;
    const TreeDims& d = h->td;
    if (q < 0 || q >= (which == 0 ? d.NI : d.NI - 1)) return SLAB_EINVAL;
    const int64_t blk = (int64_t)d.s_pad * d.s_pad;
    const bool mirror = which == 2 && !h->Tl;          // symmetric kinds: T_{q+1,q} = T_{q,q+1}^T
    const void* src = which == 0 ? h->Tb : (which == 1 || mirror ? h->To : h->Tl);
    const unsigned char* base = (const unsigned char*)src + q * blk * h->rsz2;
    std::vector<unsigned char> tmp((size_t)blk * h->rsz2);
    SLAB_CK(h, cudaMemcpyAsync(tmp.data(), base, tmp.size(), cudaMemcpyDeviceToHost, h->stream));
    SLAB_CK(h, cudaStreamSynchronize(h->stream));
    const double sc = (double)h->n * (double)h->n;
    for (int i = 0; i < d.si; ++i)
        for (int j = 0; j < d.si; ++j) {
            const int64_t e = (int64_t)i * d.s_pad + j;
            const double v = h->rsz2 == 8 ? ((const double*)tmp.data())[e] : (double)((const float*)tmp.data())[e];
            out[mirror ? (int64_t)j * d.si + i : (int64_t)i * d.si + j] = sc * v;
        }
    return SLAB_OK;
}

slab_status slab_sizes(const slab_handle* h, int64_t* unknowns, int64_t* iface_size, int* n_ifaces) {
    if (!h) return SLAB_EINVAL;
    int64_t N = 1;
    for (int i = 0; i < h->dim; ++i) N *= h->n - 1;
    if (unknowns) *unknowns = N;
    if (iface_size) *iface_size = N / (h->n - 1);
    if (n_ifaces) *n_ifaces = h->td.NI;
    return SLAB_OK;
}

int64_t slab_device_bytes(const slab_handle* h) { return h ? h->dev_bytes : 0; }

int slab_stage2_order(const slab_handle* h) {
    if (!h) return 0;
    return h->stage2 ? SLAB_STAGE2_ODDEVEN : SLAB_STAGE2_SWEEP;
}

slab_status slab_last_error(const slab_handle* h) { return h ? h->err : SLAB_EINVAL; }

}  // extern "C"

// ------------------------------------------------------------------ batches of independent problems
namespace {

// run body(i) for i < count on up to `workers` host threads (each drives its own handles' streams)
template <typename F>
slab_status run_batch(int count, int workers, F body) {
    if (count <= 0) return SLAB_OK;
    if (workers <= 0) workers = 8;
    workers = std::min(workers, count);
    int device = 0;
    cudaGetDevice(&device);
    std::atomic<int> next(0);
    std::vector<slab_status> st(count, SLAB_OK);
    auto work = [&]() {
        cudaSetDevice(device);
        for (int i = next.fetch_add(1); i < count; i = next.fetch_add(1)) st[i] = body(i);
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < workers; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < count; ++i)
        if (st[i] != SLAB_OK) return st[i];
    return SLAB_OK;
}

}  // namespace

slab_status slab_factor_batched(int count, const slab_grid* grids, const slab_coeffs* coeffs, const int* b,
                                const slab_opts* opts, int workers, slab_handle** out) {
    if (count < 0 || (count > 0 && (!grids || !coeffs || !b || !out))) return SLAB_EINVAL;
    slab_opts base;
    if (opts) base = *opts;
    else slab_default_opts(&base);
    return run_batch(count, workers, [&](int i) -> slab_status {
        out[i] = nullptr;
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return SLAB_ECUDA;
        }
        slab_opts o = base;
        o.stream = s;
        slab_handle* h = nullptr;
        const slab_status st = slab_factor(&grids[i], &coeffs[i], b[i], &o, &h);
        if (st != SLAB_OK) {
            cudaStreamDestroy(s);
            return st;
        }
        h->own_stream = 1;
        out[i] = h;
        return SLAB_OK;
    });
}

slab_status slab_solve_batched(int count, slab_handle* const* h, const double* const* f, double* const* u,
                               const int* k, double* const* relres_out, int* iters_out, int workers) {
    if (count < 0 || (count > 0 && (!h || !f || !u || !k))) return SLAB_EINVAL;
    return run_batch(count, workers, [&](int i) -> slab_status {
        return slab_solve(h[i], f[i], u[i], k[i], relres_out ? relres_out[i] : nullptr,
                          iters_out ? &iters_out[i] : nullptr);
    });
}

slab_status slab_adjoint_batched(int count, slab_handle* const* h, const double* const* dLdu,
                                 const double* const* u, double* const* lambda, double* const* dLdkappa,
                                 const int* k, int workers) {
    if (count < 0 || (count > 0 && (!h || !dLdu || !lambda || !k))) return SLAB_EINVAL;
    return run_batch(count, workers, [&](int i) -> slab_status {
        const slab_status st =
            slab_adjoint(h[i], dLdu[i], u ? u[i] : nullptr, lambda[i], dLdkappa ? dLdkappa[i] : nullptr, k[i]);
        if (h[i] && h[i]->stream) cudaStreamSynchronize(h[i]->stream);
        return st;
    });
}
