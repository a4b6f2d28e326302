// Batches of independent 2-D diffusion problems with the least-squares objective, run as CUDA
// graphs (the batched adjoint workload).
//
// Creation allocates everything once -- the factors and work areas of every problem and the
// caller-visible inputs and outputs -- from one device region, and records, per wave of
// problems, every launch of
//   coefficients, factor (Stage 1, T, Stage 2), u = A^-1 f with a fixed number of refinement
//   passes, L = ||u - t||^2 and dL/du = 2 (u - t), lambda = A^-T dL/du (same factors, A = A^T),
//   dL/dkappa = -lambda^T (dA/dkappa) u
// into one CUDA graph whose problems run on parallel branches.  A run is then one graph launch
// per wave, with no allocation, no host synchronisation and no host decision inside.  Waves run
// one after another and share the factor memory (the region holds the inputs and outputs of
// every problem plus the factors of the largest wave); the refinement count is fixed at
// creation, and the results report the relative residual each problem reached.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "slab_internal.cuh"

namespace {

constexpr int MF_BLOCKS = 256;     // partial sums of the misfit reduction

// d = 2 (u - t); part[block] = sum over the block's strided range of (u - t)^2
__global__ void __launch_bounds__(256) misfit_partial_kernel(const double* __restrict__ u,
                                                             const double* __restrict__ t, double* d, int64_t N,
                                                             double* part) {
    __shared__ double red[8];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const double e = u[i] - t[i];
        d[i] = 2.0 * e;
        acc += e * e;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// loss = sum of the partial sums, in a fixed order (one warp)
__global__ void misfit_final_kernel(const double* __restrict__ part, int nparts, double* loss) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += 32) acc += part[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) *loss = acc;
}

struct ResultPtrs {
    const unsigned* status;    // device status word of the problem's handle
    const double* nrm;         // [4]: ||f - A u||^2, ||f||^2, ||g - A lambda||^2, ||g||^2
    const double* loss;
};

// res[i] = {status, four squared norms, loss} of problem i, gathered for one host copy
__global__ void collect_kernel(const ResultPtrs* __restrict__ p, int i0, int count, double* res) {
    const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= i0 + count) return;
    double* r = res + (int64_t)i * 6;
    r[0] = (double)*p[i].status;
    for (int q = 0; q < 4; ++q) r[1 + q] = p[i].nrm[q];
    r[5] = *p[i].loss;
}

struct ProblemIO {
    double *kappa, *f, *t, *u, *lam, *d, *grad, *nrm, *loss, *part;
};

}  // namespace

struct slab_batch {
    int count = 0, wave = 0, waves = 0, branches = 0, steps = 0;
    double rtol = 1e-10;
    std::vector<int> n, b;
    std::vector<slab_handle*> h;
    std::vector<ProblemIO> io;
    void* mem = nullptr;
    size_t bytes = 0;
    SlabArena arena_io{nullptr, 0, 0};
    std::vector<SlabArena> arena_wave;  // one per wave (handles keep a pointer to theirs)
    ResultPtrs* ptrs = nullptr;         // device table (in the region)
    double* res = nullptr;              // device results [count][6] (in the region)
    std::vector<cudaGraph_t> graph;
    std::vector<cudaGraphExec_t> exec;
    std::vector<cudaStream_t> br;
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    cudaStream_t last = nullptr;        // stream of the last run
};

namespace {

slab_status take(SlabArena* A, void** p, size_t bytes) {
    const size_t off = (A->off + 255) & ~(size_t)255;
    if (A->base && off + bytes > A->cap) return SLAB_ENOMEM;
    *p = A->base + off;
    A->off = off + bytes;
    return SLAB_OK;
}

// Inputs, outputs and per-problem reduction buffers of every problem, from arena A.
slab_status carve_io(slab_batch* B, SlabArena* A) {
    B->io.assign(B->count, ProblemIO{});
    for (int i = 0; i < B->count; ++i) {
        const size_t nodes = (size_t)(B->n[i] + 1) * (B->n[i] + 1), N = (size_t)(B->n[i] - 1) * (B->n[i] - 1);
        ProblemIO& q = B->io[i];
        void* p;
        slab_status st;
#define TAKE(field, bytes) if ((st = take(A, &p, (bytes)))) return st; q.field = (double*)p
        TAKE(kappa, nodes * 8);
        TAKE(f, N * 8);
        TAKE(t, N * 8);
        TAKE(u, N * 8);
        TAKE(lam, N * 8);
        TAKE(d, N * 8);
        TAKE(grad, nodes * 8);
        TAKE(nrm, 4 * 8);
        TAKE(loss, 8);
        TAKE(part, MF_BLOCKS * 8);
#undef TAKE
    }
    void* p;
    slab_status st;
    if ((st = take(A, &p, (size_t)B->count * sizeof(ResultPtrs)))) return st;
    B->ptrs = (ResultPtrs*)p;
    if ((st = take(A, &p, (size_t)B->count * 6 * sizeof(double)))) return st;
    B->res = (double*)p;
    return SLAB_OK;
}

// Handles of wave w (factor + solve buffers for one load) from arena A.
slab_status create_wave(slab_batch* B, int w, const slab_opts& o, SlabArena* A) {
    const int i0 = w * B->wave, i1 = std::min(B->count, i0 + B->wave);
    for (int i = i0; i < i1; ++i) {
        slab_grid g{2, B->n[i]};
        slab_coeffs co{SLAB_DIFFUSION, B->io[i].kappa, nullptr, 0.0};
        slab_handle* h = nullptr;
        slab_status st = factor_create(&g, &co, B->b[i], &o, &h, A);
        if (st) return st;
        B->h[i] = h;
        h->stream = B->cap;
        if ((st = solve_prepare(h, 1))) return st;
    }
    return SLAB_OK;
}

void release_handles(slab_batch* B) {
    for (auto& h : B->h) {
        if (h) slab_destroy(h);
        h = nullptr;
    }
}

// Record the work of problem i on stream s (inside a capture).
slab_status record_problem(slab_batch* B, int i, cudaStream_t s) {
    slab_handle* h = B->h[i];
    const ProblemIO& q = B->io[i];
    h->stream = s;
    const int64_t N = h->td.N;
    slab_status st;
    if ((st = reset_scratch(h))) return st;
    if ((st = factor_launch(h, q.kappa, nullptr))) return st;
    if ((st = solve_fixed(h, q.f, q.u, 1, B->steps, q.nrm))) return st;
    misfit_partial_kernel<<<MF_BLOCKS, 256, 0, s>>>(q.u, q.t, q.d, N, q.part);
    SLAB_CK_LAUNCH(h);
    misfit_final_kernel<<<1, 32, 0, s>>>(q.part, MF_BLOCKS, q.loss);
    SLAB_CK_LAUNCH(h);
    if ((st = solve_fixed(h, q.d, q.lam, 1, B->steps, q.nrm + 2))) return st;   // A = A^T: same factors
    SLAB_CK(h, cudaMemsetAsync(q.grad, 0, (size_t)(h->n + 1) * (h->n + 1) * sizeof(double), s));
    return launch_kappa_gradient(h, q.u, q.lam, q.grad, 1);
}

// Capture wave w into a graph: problems spread over the branches (largest first, each to the
// branch with the least modelled work), forked from and joined back into the capture stream.
slab_status capture_wave(slab_batch* B, int w) {
    const int i0 = w * B->wave, i1 = std::min(B->count, i0 + B->wave);
    std::vector<int> order(i1 - i0);
    std::iota(order.begin(), order.end(), i0);
    std::sort(order.begin(), order.end(), [&](int a, int c) { return B->n[a] > B->n[c]; });
    std::vector<double> load(B->branches, 0.0);
    std::vector<std::vector<int>> lane(B->branches);
    for (int i : order) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane[k].push_back(i);
        load[k] += (double)B->n[i] * B->n[i] * B->n[i] / B->b[i];
    }
    if (cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) return SLAB_ECUDA;
    slab_status st = SLAB_OK;
    if (cudaEventRecord(B->fork, B->cap) != cudaSuccess) st = SLAB_ECUDA;
    for (int k = 0; k < B->branches && !st; ++k) {
        if (cudaStreamWaitEvent(B->br[k], B->fork, 0) != cudaSuccess) { st = SLAB_ECUDA; break; }
        for (int i : lane[k])
            if ((st = record_problem(B, i, B->br[k]))) break;
        if (!st && cudaEventRecord(B->join[k], B->br[k]) != cudaSuccess) st = SLAB_ECUDA;
        if (!st && cudaStreamWaitEvent(B->cap, B->join[k], 0) != cudaSuccess) st = SLAB_ECUDA;
    }
    if (!st) {
        collect_kernel<<<(i1 - i0 + 127) / 128, 128, 0, B->cap>>>(B->ptrs, i0, i1 - i0, B->res);
        if (cudaGetLastError() != cudaSuccess) st = SLAB_ECUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(B->cap, &g);
    if (st || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return st ? st : SLAB_ECUDA;
    }
    cudaGraphExec_t x = nullptr;
    if (cudaGraphInstantiate(&x, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    B->graph[w] = g;
    B->exec[w] = x;
    return SLAB_OK;
}

}  // namespace

extern "C" {

void slab_batch_destroy(slab_batch* B) {
    if (!B) return;
    if (B->last) cudaStreamSynchronize(B->last);
    if (B->cap) cudaStreamSynchronize(B->cap);
    for (auto x : B->exec) if (x) cudaGraphExecDestroy(x);
    for (auto g : B->graph) if (g) cudaGraphDestroy(g);
    release_handles(B);
    for (auto s : B->br) if (s) cudaStreamDestroy(s);
    for (auto e : B->join) if (e) cudaEventDestroy(e);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->mem) cudaFree(B->mem);
    delete B;
}

slab_status slab_batch_create(int count, const int* n, const int* b, const slab_opts* opts, int steps, int wave,
                              int branches, slab_batch** out) {
    if (!out) return SLAB_EINVAL;
    *out = nullptr;
    if (count <= 0 || !n || !b || steps < 0 || steps > 100 || branches < 0 || branches > 64 || wave < 0)
        return SLAB_EINVAL;
    slab_opts o;
    if (opts) o = *opts;
    else slab_default_opts(&o);
    if (o.krylov != 0) return SLAB_EUNSUPPORTED;       // the fixed-pass refinement only
    o.profile = 0;
    o.stream = nullptr;
    for (int i = 0; i < count; ++i)
        if (b[i] < 2 || n[i] < 4 || n[i] % b[i] || n[i] / b[i] < 2) return SLAB_EINVAL;
    slab_batch* B = new (std::nothrow) slab_batch();
    if (!B) return SLAB_ENOMEM;
    B->count = count;
    B->wave = wave > 0 ? std::min(wave, count) : count;
    B->waves = (count + B->wave - 1) / B->wave;
    B->branches = branches > 0 ? branches : 16;
    B->steps = steps;
    B->rtol = o.rtol;
    B->n.assign(n, n + count);
    B->b.assign(b, b + count);
    B->h.assign(count, nullptr);
    B->graph.assign(B->waves, nullptr);
    B->exec.assign(B->waves, nullptr);
    slab_status st = SLAB_OK;
    // sizing pass: offsets only (nothing is launched or touched), then one allocation.  Every arena
    // starts at offset 256, so that no buffer of the sizing pass is a null pointer.
    SlabArena io{nullptr, 256, 0};
    if ((st = carve_io(B, &io))) { slab_batch_destroy(B); return st; }
    size_t wave_max = 0;
    for (int w = 0; w < B->waves && !st; ++w) {
        SlabArena A{nullptr, 256, 0};
        st = create_wave(B, w, o, &A);
        release_handles(B);
        wave_max = std::max(wave_max, A.off);
    }
    if (st) { slab_batch_destroy(B); return st; }
    const size_t io_bytes = (io.off + 255) & ~(size_t)255;
    B->bytes = io_bytes + wave_max;
    if (cudaMalloc(&B->mem, B->bytes) != cudaSuccess) {
        cudaGetLastError();
        B->mem = nullptr;
        slab_batch_destroy(B);
        return SLAB_ENOMEM;
    }
    B->arena_io = SlabArena{(char*)B->mem, 256, io_bytes};
    if ((st = carve_io(B, &B->arena_io))) { slab_batch_destroy(B); return st; }
    std::vector<ResultPtrs> tab(count);
    for (int i = 0; i < count; ++i) tab[i] = ResultPtrs{nullptr, B->io[i].nrm, B->io[i].loss};
    if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        slab_batch_destroy(B);
        return SLAB_ECUDA;
    }
    B->br.assign(B->branches, nullptr);
    B->join.assign(B->branches, nullptr);
    for (int k = 0; k < B->branches; ++k)
        if (cudaStreamCreateWithFlags(&B->br[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->join[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            slab_batch_destroy(B);
            return SLAB_ECUDA;
        }
    // per wave: the handles in the shared factor region, then the graph; the handles' host state
    // (sizes, buffer addresses) is what the graph was recorded from, so each wave keeps its own
    B->arena_wave.assign(B->waves, SlabArena{(char*)B->mem + io_bytes, 256, wave_max});
    for (int w = 0; w < B->waves; ++w) {
        st = create_wave(B, w, o, &B->arena_wave[w]);
        const int i0 = w * B->wave, i1 = std::min(count, i0 + B->wave);
        for (int i = i0; i < i1 && !st; ++i) tab[i].status = B->h[i]->dstatus;
        if (!st) st = capture_wave(B, w);
        if (st) { slab_batch_destroy(B); return st; }
    }
    if (cudaMemcpy(B->ptrs, tab.data(), count * sizeof(ResultPtrs), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(B->res, 0, (size_t)count * 6 * sizeof(double)) != cudaSuccess ||
        cudaStreamSynchronize(B->cap) != cudaSuccess) {
        cudaGetLastError();
        slab_batch_destroy(B);
        return SLAB_ECUDA;
    }
    *out = B;
    return SLAB_OK;
}

slab_status slab_batch_buffers(slab_batch* B, int i, double** kappa, double** f, double** target, double** u,
                               double** lambda, double** grad) {
    if (!B || i < 0 || i >= B->count) return SLAB_EINVAL;
    const ProblemIO& q = B->io[i];
    if (kappa) *kappa = q.kappa;
    if (f) *f = q.f;
    if (target) *target = q.t;
    if (u) *u = q.u;
    if (lambda) *lambda = q.lam;
    if (grad) *grad = q.grad;
    return SLAB_OK;
}

slab_status slab_batch_run(slab_batch* B, void* stream) {
    if (!B) return SLAB_EINVAL;
    const cudaStream_t s = (cudaStream_t)stream;
    for (int w = 0; w < B->waves; ++w)
        if (cudaGraphLaunch(B->exec[w], s) != cudaSuccess) {
            cudaGetLastError();
            return SLAB_ECUDA;
        }
    B->last = s;
    return SLAB_OK;
}

slab_status slab_batch_results(slab_batch* B, double* loss, double* relres_u, double* relres_lambda) {
    if (!B) return SLAB_EINVAL;
    if (cudaStreamSynchronize(B->last) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    std::vector<double> r((size_t)B->count * 6);
    if (cudaMemcpy(r.data(), B->res, r.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    slab_status st = SLAB_OK;
    for (int i = 0; i < B->count; ++i) {
        const double* q = &r[(size_t)i * 6];
        const unsigned dev = (unsigned)q[0];
        const double ru = q[2] > 0 ? std::sqrt(q[1] / q[2]) : (q[1] > 0 ? INFINITY : 0.0);
        const double rl = q[4] > 0 ? std::sqrt(q[3] / q[4]) : (q[3] > 0 ? INFINITY : 0.0);
        if (loss) loss[i] = q[5];
        if (relres_u) relres_u[i] = ru;
        if (relres_lambda) relres_lambda[i] = rl;
        slab_status si = SLAB_OK;
        if (dev & SLAB_DEV_TIMEOUT) si = SLAB_ETIMEOUT;
        else if (dev & SLAB_DEV_NOTSPD) si = SLAB_ESINGULAR;
        else if (!(ru <= B->rtol) || !(rl <= B->rtol)) si = SLAB_ENOCONV;
        if (si && (!st || st == SLAB_ENOCONV)) st = si;
    }
    return st;
}

int64_t slab_batch_device_bytes(const slab_batch* B) { return B ? (int64_t)B->bytes : 0; }

}  // extern "C"
