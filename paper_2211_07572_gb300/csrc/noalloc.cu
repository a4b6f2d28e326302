// slab_residual_norms_noalloc: the FP64 stencil residual r = f - A u with the squared norms
// ||r_q||^2 and ||f_q||^2, for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not allowed -- inside a
// CUDA stream capture that must not contain allocation nodes, in a process whose memory pool
// is owned and budgeted by another framework, or in a real-time loop that forbids allocator
// calls.  Such a caller passes its own input and output buffers; the only scratch the kernel
// needs (per-block partial sums and per-group counters of the norm reduction) lives in the
// fixed file-scope arrays below, which every GPU that loads this library holds until exit.
//
// Limits and sharing rules:
//   * k * ceil((n-1)/256) * ceil((n-1)/NA_ROWS) * 2 <= NA_PART_DOUBLES (4 MiB of doubles) and
//     ceil(k/NA_Q) <= NA_MAX_GROUPS; larger requests are rejected with SLAB_EINVAL.
//   * All calls share the one scratch array, which keeps the last call's contents.  Calls
//     that overlap on the GPU (concurrent streams, or two host threads) race on it and give
//     wrong norms; serialise them.
//   * The first call on a device looks up the device address of the scratch arrays for that
//     device (a runtime query, not an allocation).  Make that first call before any stream
//     capture begins.
#include <mutex>

#include "slab_internal.cuh"

#define NA_PART_DOUBLES (1 << 19)   // 512 Ki doubles = 4 MiB of partial sums
#define NA_MAX_GROUPS 1024          // right-hand-side groups per call
#define NA_ROWS 32                  // grid rows per block
#define NA_Q 8                      // right-hand sides per group
#define NA_MAX_DEVICES 64

static __device__ __align__(256) double g_na_part[NA_PART_DOUBLES];
static __device__ __align__(256) unsigned g_na_tickets[NA_MAX_GROUPS];

namespace {

// Face coefficient of the operator between node indices a and b of the (n+1)^2 node array.
__device__ inline double na_face(int kind, const double* kappa, int64_t a, int64_t b) {
    return kind == SLAB_DIFFUSION ? 0.5 * (kappa[a] + kappa[b]) : 1.0;
}

__global__ void __launch_bounds__(256) na_residual_kernel(int n, int k, int kind, const double* __restrict__ kappa,
                                                          const double* __restrict__ c, double omega,
                                                          const double* __restrict__ u,
                                                          const double* __restrict__ f, double* r,
                                                          double* nrm_r, double* nrm_f, double* part,
                                                          unsigned* tickets) {
    const int s = n - 1;
    const int np1 = n + 1;
    const int q0 = blockIdx.z * NA_Q;
    const int nq = min(NA_Q, k - q0);
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const double n2 = (double)n * (double)n;
    const int64_t N = (int64_t)s * s;
    double rr2[NA_Q], ff2[NA_Q];
#pragma unroll
    for (int q = 0; q < NA_Q; ++q) rr2[q] = ff2[q] = 0.0;
    if (x <= s) {
        for (int yy = 0; yy < NA_ROWS; ++yy) {
            const int y = blockIdx.y * NA_ROWS + yy + 1;
            if (y > s) break;
            const int64_t P = (int64_t)y * np1 + x;
            const double fw = na_face(kind, kappa, P, P - 1), fe = na_face(kind, kappa, P, P + 1);
            const double fs = na_face(kind, kappa, P, P - np1), fn = na_face(kind, kappa, P, P + np1);
            double d = fw + fe + fs + fn;
            if (kind == SLAB_HELMHOLTZ) {
                const double wv = omega / c[P] / n;
                d -= wv * wv;
            }
            const int64_t i = (int64_t)(y - 1) * s + (x - 1);
#pragma unroll
            for (int q = 0; q < NA_Q; ++q) {
                if (q < nq) {
                    const double* uq = u + (q0 + q) * N;
                    const double uw = x > 1 ? uq[i - 1] : 0.0, ue = x < s ? uq[i + 1] : 0.0;
                    const double us = y > 1 ? uq[i - s] : 0.0, un = y < s ? uq[i + s] : 0.0;
                    const double Au = n2 * (d * uq[i] - fw * uw - fe * ue - fs * us - fn * un);
                    const double fv = f[(q0 + q) * N + i];
                    const double rv = fv - Au;
                    r[(q0 + q) * N + i] = rv;
                    rr2[q] += rv * rv;
                    ff2[q] += fv * fv;
                }
            }
        }
    }
    __shared__ double red[2][NA_Q][8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < NA_Q; ++q) {
        double a = rr2[q], b = ff2[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (l == 0) { red[0][q][w] = a; red[1][q][w] = b; }
    }
    __syncthreads();
    const int nblk = gridDim.x * gridDim.y;
    const int bid = blockIdx.y * gridDim.x + blockIdx.x;
    __shared__ bool last;
    if (threadIdx.x < 2 * NA_Q) {
        const int which = threadIdx.x / NA_Q, q = threadIdx.x % NA_Q;
        double sum = 0;
        for (int t = 0; t < 8; ++t) sum += red[which][q][t];
        if (q < nq) part[(((int64_t)(q0 + q)) * nblk + bid) * 2 + which] = sum;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(tickets + blockIdx.z, 1u) == (unsigned)(nblk - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double red2[256];
    for (int qq = 0; qq < 2 * nq; ++qq) {
        const int q = qq >> 1, which = qq & 1;
        double sum = 0;
        for (int t = threadIdx.x; t < nblk; t += blockDim.x)
            sum += __ldcg(part + (((int64_t)(q0 + q)) * nblk + t) * 2 + which);
        red2[threadIdx.x] = sum;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red2[threadIdx.x] += red2[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (which == 0) nrm_r[q0 + q] = red2[0];
            else nrm_f[q0 + q] = red2[0];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) tickets[blockIdx.z] = 0;
}

// Device addresses of the scratch arrays, looked up once per device.
struct NaScratch {
    double* part = nullptr;
    unsigned* tickets = nullptr;
    bool ready = false;
};
NaScratch g_na_dev[NA_MAX_DEVICES];
std::mutex g_na_mutex;

slab_status na_scratch_for_current_device(NaScratch* out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SLAB_ECUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return SLAB_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaScratch& sc = g_na_dev[dev];
    if (!sc.ready) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_part) != cudaSuccess) { cudaGetLastError(); return SLAB_ECUDA; }
        sc.part = (double*)p;
        if (cudaGetSymbolAddress(&p, g_na_tickets) != cudaSuccess) { cudaGetLastError(); return SLAB_ECUDA; }
        sc.tickets = (unsigned*)p;
        sc.ready = true;
    }
    *out = sc;
    return SLAB_OK;
}

}  // namespace

extern "C" slab_status slab_residual_norms_noalloc(int n, int kind, const double* kappa, const double* c,
                                                   double omega, const double* u, const double* f, double* r,
                                                   int k, double* nrm_r, double* nrm_f, void* stream) {
    if (n < 2 || k < 0 || kind < SLAB_POISSON || kind > SLAB_HELMHOLTZ) return SLAB_EINVAL;
    if (kind == SLAB_DIFFUSION && !kappa) return SLAB_EINVAL;
    if (kind == SLAB_HELMHOLTZ && !c) return SLAB_EINVAL;
    if (k == 0) return SLAB_OK;
    if (!u || !f || !r || !nrm_r || !nrm_f) return SLAB_EINVAL;
    const int s = n - 1;
    dim3 grid((s + 255) / 256, (s + NA_ROWS - 1) / NA_ROWS, (k + NA_Q - 1) / NA_Q);
    const int64_t need = (int64_t)k * grid.x * grid.y * 2;
    if (need > NA_PART_DOUBLES || grid.z > NA_MAX_GROUPS || grid.y > 65535u) return SLAB_EINVAL;
    NaScratch sc;
    slab_status st = na_scratch_for_current_device(&sc);
    if (st != SLAB_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    // the counters must start at zero; a memset is not an allocation
    if (cudaMemsetAsync(sc.tickets, 0, grid.z * sizeof(unsigned), cs) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    na_residual_kernel<<<grid, 256, 0, cs>>>(n, k, kind, kappa, c, omega, u, f, r, nrm_r, nrm_f, sc.part,
                                             sc.tickets);
    if (cudaGetLastError() != cudaSuccess) return SLAB_ECUDA;
    return SLAB_OK;
}
