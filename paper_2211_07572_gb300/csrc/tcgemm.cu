// Tensor-core product C = alpha A B^T + beta C on sm_103a (tcgen05 + TMA + TMEM), FP32 data.
//
// A is M x K and B is N x K, both row-major (K contiguous, "K-major"), optionally batched.
// Each CTA computes a 128 x BN tile of C:
//   warp 0      TMA producer: 128 x 32 and BN x 32 FP32 boxes, 128-byte swizzle, into a
//               STAGES-deep ring guarded by mbarriers (full / empty)
//   warps 4..7  split each landed FP32 element x into hi = rna_tf32(x) and lo = x - hi
//               (3xTF32 mode), fence the writes for the async proxy and arrive on conv;
//               afterwards they are the epilogue (TMEM -> registers -> global)
//   warp 1      allocates TMEM and, from one thread, issues tcgen05.mma.kind::tf32:
//               A_hi B_hi + A_hi B_lo + A_lo B_hi per K-slice of 8 (FP32-level accuracy,
//               relative error ~2^-22 per product), accumulating in TMEM (FP32)
// Every wait is bounded; a wait that runs out sets bit 2 of *err, the CTA stops issuing work,
// waits (bounded) for the copies it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "slab_internal.cuh"

namespace {

// Opt a kernel in to its dynamic shared memory once per device (idempotent, safe from several
// host threads: the batched entry points drive problems from a worker pool).
template <typename Kern>
bool ensure_smem_attr(Kern kernel, int bytes, std::atomic<uint32_t>& done) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    const uint32_t bit = 1u << (dev & 31);
    if (done.load(std::memory_order_acquire) & bit) return true;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess) return false;
    done.fetch_or(bit, std::memory_order_acq_rel);
    return true;
}

// Streaming multiprocessors of the current device (cached per device).
int num_sms() {
    static std::atomic<int> cache[32];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    std::atomic<int>& c = cache[dev & 31];
    int v = c.load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 148;
    c.store(v, std::memory_order_relaxed);
    return v;
}

constexpr int BM = 128;
constexpr int BK = 32;                 // 32 FP32 = one 128-byte swizzle row
constexpr uint32_t WAIT_LIMIT = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
// 32 lanes x 32 columns of 32-bit TMEM data: this thread's lane, columns [col, col+32)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);      // start address (16-byte units)
    d |= (uint64_t)1 << 16;                         // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)2 << 61;                         // swizzle mode: 128 B
    return d;
}
// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int BN, bool SPLIT>
struct TcCfg {
    static constexpr int STAGES = SPLIT ? (BN <= 32 ? 5 : (BN <= 64 ? 4 : 3)) : 5;   // as many as fit in 227 KB
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = BN * BK * 4;
    static constexpr int STAGE_BYTES = (SPLIT ? 2 : 1) * (A_BYTES + B_BYTES);
    static constexpr int EPI_BYTES = 4 * 32 * 33 * 4;            // per-warp 32 x 32 staging tiles
    static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024;   // + alignment slack
};

template <int BN, bool SPLIT>
__global__ void __launch_bounds__(256, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                   int K, float alpha, float beta, float* C, int64_t ldc, int64_t c_bstride, int transC,
                   int lower_only, int triA, int ksplit, float* part, unsigned* err) {
    using Cfg = TcCfg<BN, SPLIT>;
    constexpr int STAGES = Cfg::STAGES;
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ uint64_t full_bar[STAGES], conv_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    // blockIdx.z = batch index * ksplit + K split; split zs covers K range [zs K/ksplit, (zs+1) K/ksplit)
    const int bn = blockIdx.x, bm = blockIdx.y;
    const int zs = (int)blockIdx.z % ksplit;
    const int bz = (int)blockIdx.z / ksplit;
    if (lower_only && bn * BN >= (bm + 1) * BM) return;        // tile strictly above the diagonal
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // K range of this split, cut to the nonzero part of a triangular A (all bounds multiples of BK)
    int k0 = zs * (K / ksplit), k1 = k0 + K / ksplit;
    if (triA == 1) k1 = min(k1, (bm + 1) * BM);
    else if (triA == 2) k0 = max(k0, bm * BM);
    const int nk = k1 > k0 ? (k1 - k0) / BK : 0;        // 0: the tile's product is zero
    uint8_t* base = (uint8_t*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
    auto a_hi = [&](int s) { return base + s * Cfg::STAGE_BYTES; };
    auto b_hi = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES; };
    auto a_lo = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES + Cfg::B_BYTES; };
    auto b_lo = [&](int s) { return base + s * Cfg::STAGE_BYTES + 2 * Cfg::A_BYTES + Cfg::B_BYTES; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&conv_bar[s], 128);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {                                         // TMA producer
            int issued = 0;
            for (int kt = 0; kt < nk && !abort_flag; ++kt) {
                const int s = kt % STAGES;
                if (kt >= STAGES && !mbar_wait(&empty_bar[s], ((kt / STAGES) - 1) & 1)) {
                    abort_flag = 1;
                    atomicOr(err, 2u);
                    break;
                }
                mbar_expect_tx(&full_bar[s], Cfg::A_BYTES + Cfg::B_BYTES);
                tma_load_3d(a_hi(s), &tmA, &full_bar[s], k0 + kt * BK, bm * BM, bz);
                tma_load_3d(b_hi(s), &tmB, &full_bar[s], k0 + kt * BK, bn * BN, bz);
                issued = kt + 1;
            }
            if (abort_flag)                                     // let the copies already issued land
                for (int kt = (issued > STAGES ? issued - STAGES : 0); kt < issued; ++kt)
                    mbar_wait(&full_bar[kt % STAGES], (kt / STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                         // MMA issuer
            constexpr uint32_t idesc = idesc_tf32(BM, BN);
            bool ok = true;
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % STAGES;
                if (abort_flag || !mbar_wait(SPLIT ? &conv_bar[s] : &full_bar[s], (kt / STAGES) & 1)) {
                    abort_flag = 1;
                    atomicOr(err, 2u);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint64_t dah = sdesc_sw128(smem_u32(a_hi(s))), dbh = sdesc_sw128(smem_u32(b_hi(s)));
                const uint64_t dal = sdesc_sw128(smem_u32(a_lo(s))), dbl = sdesc_sw128(smem_u32(b_lo(s)));
#pragma unroll
                for (int kk = 0; kk < BK / 8; ++kk) {            // 8 TF32 = 32 bytes per MMA
                    const uint64_t off = (uint64_t)(kk * 2);
                    mma_tf32(tmem, dah + off, dbh + off, idesc, (kt | kk) != 0);
                    if (SPLIT) {
                        mma_tf32(tmem, dah + off, dbl + off, idesc, 1);
                        mma_tf32(tmem, dal + off, dbh + off, idesc, 1);
                    }
                }
                mma_commit(&empty_bar[s]);
            }
            if (ok && nk > 0) mma_commit(&done_bar);
        }
    } else if (warp >= 4) {
        if (SPLIT) {                                             // hi/lo split of each landed stage
            const int t = threadIdx.x - 128;
            for (int kt = 0; kt < nk; ++kt) {
                const int s = kt % STAGES;
                if (abort_flag || !mbar_wait(&full_bar[s], (kt / STAGES) & 1)) {
                    abort_flag = 1;
                    atomicOr(err, 2u);
                    break;
                }
                float4* ah = reinterpret_cast<float4*>(a_hi(s));
                float4* al = reinterpret_cast<float4*>(a_lo(s));
                for (int e = t; e < Cfg::A_BYTES / 16; e += 128) {
                    float4 x = ah[e], hi, lo;
                    float* px = &x.x; float* ph = &hi.x; float* pl = &lo.x;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t hb;
                        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(px[q]));
                        ph[q] = __uint_as_float(hb);
                        pl[q] = px[q] - ph[q];
                    }
                    ah[e] = hi;
                    al[e] = lo;
                }
                float4* bh = reinterpret_cast<float4*>(b_hi(s));
                float4* bl = reinterpret_cast<float4*>(b_lo(s));
                for (int e = t; e < Cfg::B_BYTES / 16; e += 128) {
                    float4 x = bh[e], hi, lo;
                    float* px = &x.x; float* ph = &hi.x; float* pl = &lo.x;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint32_t hb;
                        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(px[q]));
                        ph[q] = __uint_as_float(hb);
                        pl[q] = px[q] - ph[q];
                    }
                    bh[e] = hi;
                    bl[e] = lo;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&conv_bar[s]);
            }
        }
        // epilogue: TMEM lanes 32*(warp-4) .. +31 are rows of the tile
        const bool ok = !abort_flag && (nk == 0 || mbar_wait(&done_bar, 0));
        if (!ok) {
            abort_flag = 1;
            atomicOr(err, 2u);
        } else {
            tc_fence_after();
            const int rw = warp - 4;
            const int row = bm * BM + rw * 32 + lane;
            float* Cb = C + (int64_t)bz * c_bstride;
            float* stg = reinterpret_cast<float*>(base + STAGES * Cfg::STAGE_BYTES) + rw * 32 * 33;
#pragma unroll 1
            for (int cc = 0; cc < BN / 32; ++cc) {
                float v[32];
                if (nk > 0) tmem_ld32(tmem + ((uint32_t)(rw * 32) << 16) + (uint32_t)(cc * 32), v);
                else
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0.f;
                if (!transC && ksplit == 1) {
                    // row-major C: stage the 32 x 32 block, then each lane walks a column of it so
                    // a warp instruction covers 32 consecutive floats of one row of C; all 32 old
                    // values are loaded before any store so the loads overlap
#pragma unroll
                    for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
                    __syncwarp();
                    const int col = bn * BN + cc * 32 + lane;
                    const int row0 = bm * BM + rw * 32;
                    float old[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r)
                        old[r] = (beta != 0.f && row0 + r < M && col < N) ? Cb[(int64_t)(row0 + r) * ldc + col] : 0.f;
#pragma unroll
                    for (int r = 0; r < 32; ++r)
                        if (row0 + r < M && col < N)
                            Cb[(int64_t)(row0 + r) * ldc + col] = alpha * stg[r * 33 + lane] + beta * old[r];
                    __syncwarp();
                    continue;
                }
                if (row < M) {
                    if (ksplit > 1) {                            // raw partial sums, reduced later
                        float* pb = part + (int64_t)blockIdx.z * M * N;   // [batch][ksplit][M N]
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = bn * BN + cc * 32 + j;
                            if (col < N) pb[transC ? (int64_t)col * M + row : (int64_t)row * N + col] = v[j];
                        }
                    } else {                                     // C^T: lanes write consecutive rows
                        float old[32];
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = bn * BN + cc * 32 + j;
                            old[j] = (beta != 0.f && col < N) ? Cb[(int64_t)col * ldc + row] : 0.f;
                        }
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const int col = bn * BN + cc * 32 + j;
                            if (col < N) Cb[(int64_t)col * ldc + row] = alpha * v[j] + beta * old[j];
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, BN);
    }
}

// C_b = alpha sum_s part[b][s] + beta C_b for the batch matrices b (sC apart); part laid out like C
// (transC: [N][M], else [M][N]); the splits are added in a fixed order.
__global__ void splitk_reduce_kernel(int M, int N, int ks, const float* __restrict__ part, float alpha, float beta,
                                     float* C, int64_t ldc, int transC, int64_t sC, int batch) {
    pdl_wait();
    pdl_trigger();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)M * N;
    if (g >= tot * batch) return;
    const int64_t b = g / tot, e = g % tot;
    const float* pb = part + b * ks * tot + e;
    float v = 0.f;
    for (int s = 0; s < ks; ++s) v += pb[(int64_t)s * tot];
    int64_t idx;
    if (transC) idx = (e / M) * ldc + (e % M);          // e = col * M + row
    else idx = (e / N) * ldc + (e % N);                 // e = row * N + col
    float* Cb = C + b * sC;
    Cb[idx] = alpha * v + (beta != 0.f ? beta * Cb[idx] : 0.f);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn lookup_encode_fn() {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return (EncodeTiledFn)p;
    return nullptr;
}

EncodeTiledFn encode_fn() {
    static const EncodeTiledFn fn = lookup_encode_fn();   // thread-safe one-time initialisation
    return fn;
}

// rows x cols row-major FP32 matrix (leading dimension ld elements), batch matrices bstride apart
bool make_map(CUtensorMap* m, const float* ptr, int64_t rows, int64_t cols, int64_t ld, int batch, int64_t bstride,
              int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)(batch > 1 ? bstride : rows * ld) * 4};
    cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)ptr, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, bool SPLIT>
slab_status launch_tc(cudaStream_t st, const TcGemmArgs& g, unsigned* err) {
    CUtensorMap ta, tb;
    if (!make_map(&ta, g.A, g.M, g.K, g.lda, g.batch, g.sA, BM)) return SLAB_ECUDA;
    if (!make_map(&tb, g.B, g.N, g.K, g.ldb, g.batch, g.sB, BN)) return SLAB_ECUDA;
    const int smem = TcCfg<BN, SPLIT>::SMEM;
    static std::atomic<uint32_t> attr_done(0);
    if (!ensure_smem_attr(tc_gemm_kernel<BN, SPLIT>, smem, attr_done)) return SLAB_ECUDA;
    const int ks = g.ksplit > 1 ? g.ksplit : 1;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, ks * g.batch);
    if (launch_pdl(tc_gemm_kernel<BN, SPLIT>, grid, dim3(256), (size_t)smem, st, ta, tb, g.M, g.N, g.K, g.alpha, g.beta,
                   g.C, g.ldc, g.sC, g.transC, g.lower_only, g.triA, ks, g.part, err) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    if (ks > 1) {
        const int64_t tot = (int64_t)g.M * g.N * g.batch;
        if (launch_pdl(splitk_reduce_kernel, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, g.M, g.N, ks,
                       (const float*)g.part, g.alpha, g.beta, g.C, g.ldc, g.transC, g.sC, g.batch) != cudaSuccess) {
            cudaGetLastError();
            return SLAB_ECUDA;
        }
    }
    return SLAB_OK;
}


// ------------------------------------------------------------------ FP64-accurate product (integer slices)
// C (FP64) += alpha A B^T for FP64 A (M x K) and B (N x K), K <= 64.  Every row of A (column of
// B^T) is scaled by a power of two into (-1, 1) and cut into OZ_S slices of 7 bits:
//   A[i][k] = 2^ea_i sum_s a_s[i][k] 2^{-7(s+1)},  |a_s| <= 127 integers (exact in TF32),
// so every slice product a_s b_t^T is an exact TF32 tensor-core product and the sum over
// K <= 64 (below 2^20) and over the at most OZ_S pairs of one level d = s + t (below 2^23) is
// exact in the FP32 accumulator.  Levels d < OZ_S are kept (the neglected ones are below
// 2^{-7 OZ_S} of |A| |B|); the epilogue adds the levels in FP32 pairs (hi + lo, ~2^-48) and
// updates C in FP64.  Tile 128 x 64; TMEM holds the OZ_S level accumulators (64 columns each).
constexpr int OZ_S = 8;
constexpr int OZ_BN = 64;

struct OzCfg {
    static constexpr int A_BYTES = BM * BK * 4;
    static constexpr int B_BYTES = OZ_BN * BK * 4;
    static constexpr int CHUNK_BYTES = OZ_S * (A_BYTES + B_BYTES);     // every slice of one K-chunk
    static constexpr int SMEM = CHUNK_BYTES + 1024;
};

__global__ void __launch_bounds__(256, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                      int K, double alpha, const int* __restrict__ ea, const int* __restrict__ eb, double* C,
                      int64_t ldc, int lower_only, unsigned* err) {
    extern __shared__ __align__(1024) uint8_t oz_smem[];
    __shared__ uint64_t full_bar[OZ_S], mma_bar;          // full_bar[s]: slice s of A and of B landed
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;
    const int bn = blockIdx.x, bm = blockIdx.y;
    if (lower_only && bn * OZ_BN >= (bm + 1) * BM) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K / BK;
    uint8_t* base = (uint8_t*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
    auto a_sl = [&](int sl) { return base + sl * OzCfg::A_BYTES; };
    auto b_sl = [&](int sl) { return base + OZ_S * OzCfg::A_BYTES + sl * OzCfg::B_BYTES; };
    if (threadIdx.x == 0) {
        for (int sl = 0; sl < OZ_S; ++sl) mbar_init(&full_bar[sl], 1);
        mbar_init(&mma_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, OZ_S * OZ_BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    int last_issued = -1;                                                // (warp 0, lane 0)
    // one K-chunk at a time: TMA of every slice, then every slice pair of every level
    for (int kt = 0; kt < nk; ++kt) {
        if (warp == 0 && lane == 0 && !abort_flag) {
            if (kt > 0 && !mbar_wait(&mma_bar, (kt - 1) & 1)) {          // previous chunk's MMAs read the buffer
                abort_flag = 1;
                atomicOr(err, 2u);
            } else {
                for (int sl = 0; sl < OZ_S; ++sl) {                     // slice by slice: MMAs start early
                    mbar_expect_tx(&full_bar[sl], OzCfg::A_BYTES + OzCfg::B_BYTES);
                    tma_load_3d(a_sl(sl), &tmA, &full_bar[sl], kt * BK, bm * BM, sl);
                    tma_load_3d(b_sl(sl), &tmB, &full_bar[sl], kt * BK, bn * OZ_BN, sl);
                }
                last_issued = kt;
            }
        }
        if (warp == 1 && lane == 0) {
            // when slice s has landed, issue every pair (i, s) and (s, j), i <= s, j < s, of a kept level
            constexpr uint32_t idesc = idesc_tf32(BM, OZ_BN);
            const uint64_t da0 = sdesc_sw128(smem_u32(a_sl(0))), db0 = sdesc_sw128(smem_u32(b_sl(0)));
            uint32_t started = kt > 0 ? 0xFFu : 0u;                  // levels already written this tile
            bool ok = !abort_flag;
            for (int sl = 0; sl < OZ_S && ok; ++sl) {
                if (!mbar_wait(&full_bar[sl], kt & 1)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                for (int pr = 0; pr < 2 * sl + 1; ++pr) {
                    const int sa = pr <= sl ? pr : sl, sb = pr <= sl ? sl : pr - sl - 1;   // (i, s) then (s, j)
                    const int d = sa + sb;
                    if (d >= OZ_S) continue;
                    // slice tiles are OzCfg::A_BYTES / B_BYTES apart: advance the descriptors' addresses
                    const uint64_t da = da0 + (uint64_t)(sa * (OzCfg::A_BYTES >> 4));
                    const uint64_t db = db0 + (uint64_t)(sb * (OzCfg::B_BYTES >> 4));
                    const uint32_t acc_col = tmem + (uint32_t)(d * OZ_BN);
#pragma unroll
                    for (int kk = 0; kk < BK / 8; ++kk) {
                        const uint64_t off = (uint64_t)(kk * 2);
                        mma_tf32(acc_col, da + off, db + off, idesc, ((started >> d) & 1u) || kk > 0 ? 1u : 0u);
                    }
                    started |= 1u << d;
                }
            }
            if (!ok) {
                abort_flag = 1;
                atomicOr(err, 2u);
            } else {
                mma_commit(&mma_bar);
            }
        }
        __syncthreads();
    }
    // after an abort, let the copies already issued land before the CTA's shared memory is released
    if (warp == 0 && lane == 0 && abort_flag && last_issued >= 0)
        for (int sl = 0; sl < OZ_S; ++sl) mbar_wait(&full_bar[sl], last_issued & 1);
    // the last chunk's commit (parity (nk-1) & 1) marks every accumulator complete
    if (warp >= 4) {
        bool ok = !abort_flag && mbar_wait(&mma_bar, (nk - 1) & 1);
        if (!ok) {
            abort_flag = 1;
            atomicOr(err, 2u);
        } else {
            tc_fence_after();
            const int rw = warp - 4;
            const int row = bm * BM + rw * 32 + lane;
            const uint32_t tl = (uint32_t)(rw * 32) << 16;
#pragma unroll 1
            for (int cc = 0; cc < OZ_BN / 32; ++cc) {
                // the 32 old values of C first, so their loads overlap the level sums below
                double cold[32];
                const int col0 = bn * OZ_BN + cc * 32;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    cold[j] = (row < M && col0 + j < N) ? C[(int64_t)row * ldc + col0 + j] : 0.0;
                float hi[32], lo[32], v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) { hi[j] = 0.f; lo[j] = 0.f; }
#pragma unroll 1
                for (int d = OZ_S - 1; d >= 0; --d) {                    // small levels first
                    tmem_ld32(tmem + tl + (uint32_t)(d * OZ_BN + cc * 32), v);
                    const float sc = __int_as_float((127 - 7 * d) << 23);          // 2^{-7d}, exact
#pragma unroll
                    for (int j = 0; j < 32; ++j) {                       // (hi, lo) += v 2^{-7d}, two-sum
                        const float a = v[j] * sc;
                        const float s2 = hi[j] + a;
                        const float bb = s2 - hi[j];
                        lo[j] += (hi[j] - (s2 - bb)) + (a - bb);
                        hi[j] = s2;
                    }
                }
                if (row < M) {
                    // C += alpha 2^{ea + eb - 14} (hi + lo): the power of two is applied in FP32 (exact
                    // while in range, checked), so the FP64 work per element is two conversions and
                    // two additions
                    const int er = ea[row] - 14;
                    double* crow = C + (int64_t)row * ldc;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = bn * OZ_BN + cc * 32 + j;
                        if (col < N) {
                            const int ex = er + eb[col];
                            double c = cold[j];
                            if (ex > -60 && ex < 60 && (alpha == 1.0 || alpha == -1.0)) {
                                const float sc = alpha < 0 ? -__int_as_float((127 + ex) << 23)
                                                           : __int_as_float((127 + ex) << 23);   // exact
                                c += (double)(hi[j] * sc);
                                c += (double)(lo[j] * sc);
                            } else {
                                c += alpha * ldexp((double)hi[j] + (double)lo[j], ex);
                            }
                            crow[col] = c;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, OZ_S * OZ_BN);
    }
}

// slices of the rows of X (rows x K, leading dimension ldx): out[s][r][k] (FP32 integers), e[r]
__global__ void ozaki_split_kernel(const double* __restrict__ X, int64_t ldx, int rows, int K, float* out, int* e) {
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const double* xr = X + (int64_t)r * ldx;
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(xr[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int ex = 0;
    if (mx > 0.0) frexp(mx, &ex);                                    // mx < 2^ex
    if (lane == 0) e[r] = ex;
    for (int k = lane; k < K; k += 32) {
        const double x = xr[k];
        const long long q = __double2ll_rz(fabs(ldexp(x, 7 * OZ_S - ex)));   // |x| 2^{56-ex} < 2^56
        const float sg = x < 0.0 ? -1.f : 1.f;
#pragma unroll
        for (int sl = 0; sl < OZ_S; ++sl) {
            const int a = (int)((q >> (7 * (OZ_S - 1 - sl))) & 127);
            out[((int64_t)sl * rows + r) * K + k] = sg * (float)a;
        }
    }
}

// ------------------------------------------------------------------ FP32-accurate product on FP16 MMAs
// C = alpha A B^T + beta C for FP32 A (M x K) and B (N x K) with K % 64 == 0.  A pre-pass scales
// every row of A and B by a power of two, x = 2^e_r x', |x'| < 1 (e_r from the row's largest
// magnitude), and splits x' = hi + lo with hi = fp16(x') and lo = fp16(x' - hi): FP16 keeps 11
// significant bits, as TF32 does, so hi + lo carries x' to about 2^-22 (below 2^-24 of the row's
// largest magnitude where lo is subnormal).  The kernel accumulates A_hi B_hi + A_hi B_lo +
// A_lo B_hi in FP32 (TMEM) on tcgen05.mma.kind::f16, twice the TF32 rate and half the shared-memory
// bytes per multiply-add, with no conversion work inside the kernel; the epilogue applies
// alpha 2^(ea_i + eb_j).  Same warp roles and bounded waits as tc_gemm_kernel, minus the split warps.
constexpr int BK16 = 64;               // 64 FP16 = one 128-byte swizzle row

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// Instruction descriptor, kind::f16: D = F32, A = B = F16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int BN>
struct F16Cfg {
    static constexpr int A_BYTES = BM * BK16 * 2;
    static constexpr int B_BYTES = BN * BK16 * 2;
    static constexpr int STAGE_BYTES = 2 * (A_BYTES + B_BYTES);   // hi and lo of A and B
    // ring depth: 192 KB of operands in flight for BN = 128 and 256 (3 x 64 KB, 2 x 96 KB)
    static constexpr int STAGES = BN == 256 ? 2 : (BN == 128 ? 3 : 4);
    static constexpr int EPI_BYTES = 4 * 32 * 33 * 4;
    static constexpr int SMEM = STAGES * STAGE_BYTES + EPI_BYTES + 1024;
};

// One warp per row: e_r, then hi / lo (FP16, [rows][K] per batch matrix, rows * K apart).
__global__ void split16_kernel(const float* __restrict__ X, int64_t ldx, int64_t sx, int rows, int K, __half* hi,
                               __half* lo, int* ex) {
    pdl_wait();
    pdl_trigger();
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const int64_t bz = blockIdx.y;
    const float* xr = X + bz * sx + (int64_t)r * ldx;
    float mx = 0.f;
    for (int k = 4 * lane; k < K; k += 128) {
        const float4 v = *reinterpret_cast<const float4*>(xr + k);
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &e);                  // mx < 2^e
    if (lane == 0) ex[bz * rows + r] = e;
    __half* hr = hi + (bz * rows + r) * (int64_t)K;
    __half* lr = lo + (bz * rows + r) * (int64_t)K;
    for (int k = 4 * lane; k < K; k += 128) {
        const float4 v = *reinterpret_cast<const float4*>(xr + k);
        const float x[4] = {ldexpf(v.x, -e), ldexpf(v.y, -e), ldexpf(v.z, -e), ldexpf(v.w, -e)};
        __half h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            h[q] = __float2half_rn(x[q]);
            l[q] = __float2half_rn(x[q] - __half2float(h[q]));
        }
        *reinterpret_cast<__half2*>(hr + k) = __halves2half2(h[0], h[1]);
        *reinterpret_cast<__half2*>(hr + k + 2) = __halves2half2(h[2], h[3]);
        *reinterpret_cast<__half2*>(lr + k) = __halves2half2(l[0], l[1]);
        *reinterpret_cast<__half2*>(lr + k + 2) = __halves2half2(l[2], l[3]);
    }
}

// Persistent: grid = min(tiles, SMs), CTA c takes tiles c, c + grid, ... (row-major over
// (batch, tile row, tile column); with lower_only the tiles strictly above the diagonal are left
// out of the sequence by every role alike).  The smem ring runs on across tiles (stage counter
// it), the accumulator alternates between two TMEM buffers of BN columns (tile counter tl):
// the MMA warp fills buffer tl & 1 while the epilogue warps drain the other one.
//   full[s] / empty[s]: TMA landed / MMAs done reading stage s  (phase (it / STAGES) & 1)
//   acc_full[b]: MMAs of the tile in buffer b done (commit); acc_empty[b]: its epilogue done
//   (128 arrivals), both in phase (tl / 2) & 1.
template <int BN>
__global__ void __launch_bounds__(256, 1)
    tc_f16x3_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int M, int N,
                    int K, int batch, float alpha, float beta, float* C, int64_t ldc, int64_t c_bstride,
                    const int* __restrict__ ea, const int* __restrict__ eb, int64_t eb_bstride, int transC,
                    int lower_only, unsigned* err) {
    using Cfg = F16Cfg<BN>;
    constexpr int STAGES = Cfg::STAGES;
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K / BK16;
    const int tn = (N + BN - 1) / BN, tm = (M + BM - 1) / BM;
    const int64_t ntiles = (int64_t)batch * tm * tn;
    // tile id -> (bz, bm, bn); false for a tile strictly above the diagonal when lower_only
    auto tile_of = [&](int64_t id, int& bz, int& bm, int& bn) {
        bn = (int)(id % tn);
        const int64_t r = id / tn;
        bm = (int)(r % tm);
        bz = (int)(r / tm);
        return !(lower_only && bn * BN >= (bm + 1) * BM);
    };
    uint8_t* base = (uint8_t*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
    auto a_hi = [&](int s) { return base + s * Cfg::STAGE_BYTES; };
    auto b_hi = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES; };
    auto a_lo = [&](int s) { return base + s * Cfg::STAGE_BYTES + Cfg::A_BYTES + Cfg::B_BYTES; };
    auto b_lo = [&](int s) { return base + s * Cfg::STAGE_BYTES + 2 * Cfg::A_BYTES + Cfg::B_BYTES; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], 128);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_slot, 2 * BN);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {                                         // TMA producer
            int64_t it = 0, issued = 0;
            for (int64_t id = blockIdx.x; id < ntiles && !abort_flag; id += gridDim.x) {
                int bz, bm, bn;
                if (!tile_of(id, bz, bm, bn)) continue;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = (int)(it % STAGES);
                    if (it >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((it / STAGES) - 1) & 1)) {
                        abort_flag = 1;
                        atomicOr(err, 2u);
                        break;
                    }
                    mbar_expect_tx(&full_bar[s], Cfg::STAGE_BYTES);
                    tma_load_3d(a_hi(s), &tmAh, &full_bar[s], kt * BK16, bm * BM, bz);
                    tma_load_3d(a_lo(s), &tmAl, &full_bar[s], kt * BK16, bm * BM, bz);
                    tma_load_3d(b_hi(s), &tmBh, &full_bar[s], kt * BK16, bn * BN, bz);
                    tma_load_3d(b_lo(s), &tmBl, &full_bar[s], kt * BK16, bn * BN, bz);
                    issued = it + 1;
                }
            }
            if (abort_flag)                                     // let the copies already issued land
                for (int64_t q = (issued > STAGES ? issued - STAGES : 0); q < issued; ++q)
                    mbar_wait(&full_bar[q % STAGES], (uint32_t)(q / STAGES) & 1);
        }
    } else if (warp == 1) {
        if (lane == 0) {                                         // MMA issuer
            constexpr uint32_t idesc = idesc_f16(BM, BN);
            int64_t it = 0, tl = 0;
            for (int64_t id = blockIdx.x; id < ntiles; id += gridDim.x) {
                int bz, bm, bn;
                if (!tile_of(id, bz, bm, bn)) continue;
                const int buf = (int)(tl & 1);
                if (abort_flag ||
                    (tl >= 2 && !mbar_wait(&acce_bar[buf], (uint32_t)((tl / 2) - 1) & 1))) {
                    abort_flag = 1;
                    atomicOr(err, 2u);
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
                bool ok = true;
                for (int kt = 0; kt < nk; ++kt, ++it) {
                    const int s = (int)(it % STAGES);
                    if (abort_flag || !mbar_wait(&full_bar[s], (uint32_t)(it / STAGES) & 1)) {
                        abort_flag = 1;
                        atomicOr(err, 2u);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dah = sdesc_sw128(smem_u32(a_hi(s))), dbh = sdesc_sw128(smem_u32(b_hi(s)));
                    const uint64_t dal = sdesc_sw128(smem_u32(a_lo(s))), dbl = sdesc_sw128(smem_u32(b_lo(s)));
#pragma unroll
                    for (int kk = 0; kk < BK16 / 16; ++kk) {     // 16 FP16 = 32 bytes per MMA
                        const uint64_t off = (uint64_t)(kk * 2);
                        mma_f16(acc, dah + off, dbh + off, idesc, (kt | kk) != 0);
                        mma_f16(acc, dah + off, dbl + off, idesc, 1);
                        mma_f16(acc, dal + off, dbh + off, idesc, 1);
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&accf_bar[buf]);
                ++tl;
            }
        }
    } else if (warp >= 4) {
        // epilogue: TMEM lanes 32*(warp-4) .. +31 are rows of the tile
        const int rw = warp - 4;
        float* stg = reinterpret_cast<float*>(base + STAGES * Cfg::STAGE_BYTES) + rw * 32 * 33;
        int64_t tl = 0;
        for (int64_t id = blockIdx.x; id < ntiles; id += gridDim.x) {
            int bz, bm, bn;
            if (!tile_of(id, bz, bm, bn)) continue;
            const int buf = (int)(tl & 1);
            if (abort_flag || !mbar_wait(&accf_bar[buf], (uint32_t)(tl / 2) & 1)) {
                abort_flag = 1;
                atomicOr(err, 2u);
                break;
            }
            tc_fence_after();
            const int row = bm * BM + rw * 32 + lane;
            const int row0 = bm * BM + rw * 32;
            float* Cb = C + (int64_t)bz * c_bstride;
            const int* ebz = eb + (int64_t)bz * eb_bstride;
            const float sa = row < M ? ldexpf(alpha, ea[(int64_t)bz * M + row]) : 0.f;   // this lane's row
#pragma unroll 1
            for (int cc = 0; cc < BN / 32; ++cc) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(rw * 32) << 16) + (uint32_t)(buf * BN + cc * 32), v);
                if (!transC) {
                    // row-major C: stage the 32 x 32 block (row scale applied), then each lane
                    // walks a column of it (column scale applied); old values loaded before stores
#pragma unroll
                    for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j] * sa;
                    __syncwarp();
                    const int col = bn * BN + cc * 32 + lane;
                    const float sb = col < N ? ldexpf(1.f, ebz[col]) : 0.f;
                    float old[32];
#pragma unroll
                    for (int r = 0; r < 32; ++r)
                        old[r] = (beta != 0.f && row0 + r < M && col < N) ? Cb[(int64_t)(row0 + r) * ldc + col] : 0.f;
#pragma unroll
                    for (int r = 0; r < 32; ++r)
                        if (row0 + r < M && col < N)
                            Cb[(int64_t)(row0 + r) * ldc + col] = stg[r * 33 + lane] * sb + beta * old[r];
                    __syncwarp();
                    continue;
                }
                if (row < M) {                                   // C^T: lanes write consecutive rows
                    float old[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = bn * BN + cc * 32 + j;
                        old[j] = (beta != 0.f && col < N) ? Cb[(int64_t)col * ldc + row] : 0.f;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = bn * BN + cc * 32 + j;
                        if (col < N) Cb[(int64_t)col * ldc + row] = v[j] * sa * ldexpf(1.f, ebz[col]) + beta * old[j];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acce_bar[buf]);                          // this thread's reads of the buffer are done
            ++tl;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * BN);
    }
}

// rows x cols row-major FP16 matrices, batch of them rows * cols apart
bool make_map16(CUtensorMap* m, const __half* ptr, int64_t rows, int64_t cols, int batch, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)(rows * cols) * 2};
    cuuint32_t box[3] = {(cuuint32_t)BK16, (cuuint32_t)box_rows, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 3, (void*)ptr, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <int BN>
slab_status launch_f16x3(cudaStream_t st, const TcGemmArgs& g, unsigned* err) {
    const bool shared = f16x3_shared(g);
    const int64_t b = g.batch, K = g.K;
    const int64_t rB = shared ? g.M : g.N;                 // rows of the split that serves B
    uint8_t* w = (uint8_t*)g.w16;
    __half* Ah = (__half*)w;                 w += align256((size_t)b * g.M * K * 2);
    __half* Al = (__half*)w;                 w += align256((size_t)b * g.M * K * 2);
    __half* Bh = Ah;
    __half* Bl = Al;
    if (!shared) {
        Bh = (__half*)w;                     w += align256((size_t)b * g.N * K * 2);
        Bl = (__half*)w;                     w += align256((size_t)b * g.N * K * 2);
    }
    int* ea = (int*)w;                       w += align256((size_t)b * g.M * 4);
    int* eb = shared ? ea : (int*)w;
    if (launch_pdl(split16_kernel, dim3((unsigned)((g.M + 7) / 8), (unsigned)b), dim3(256), 0, st, g.A, g.lda, g.sA,
                   g.M, g.K, Ah, Al, ea) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    if (!shared &&
        launch_pdl(split16_kernel, dim3((unsigned)((g.N + 7) / 8), (unsigned)b), dim3(256), 0, st, g.B, g.ldb, g.sB,
                   g.N, g.K, Bh, Bl, eb) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    CUtensorMap tah, tal, tbh, tbl;
    if (!make_map16(&tah, Ah, g.M, K, g.batch, BM) || !make_map16(&tal, Al, g.M, K, g.batch, BM) ||
        !make_map16(&tbh, Bh, rB, K, g.batch, BN) || !make_map16(&tbl, Bl, rB, K, g.batch, BN))
        return SLAB_ECUDA;
    const int smem = F16Cfg<BN>::SMEM;
    static std::atomic<uint32_t> attr_done(0);
    if (!ensure_smem_attr(tc_f16x3_kernel<BN>, smem, attr_done)) return SLAB_ECUDA;
    const int64_t tiles = (int64_t)g.batch * ((g.M + BM - 1) / BM) * ((g.N + BN - 1) / BN);
    const int grid = (int)std::min<int64_t>(tiles, num_sms());
    if (launch_pdl(tc_f16x3_kernel<BN>, dim3(grid), dim3(256), (size_t)smem, st, tah, tal, tbh, tbl, g.M, g.N, g.K,
                   g.batch, g.alpha, g.beta, g.C, g.ldc, g.sC, (const int*)ea, (const int*)eb, rB, g.transC,
                   g.lower_only, err) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ECUDA;
    }
    return SLAB_OK;
}

}  // namespace

// 128 x 256 tiles halve the B-operand traffic per flop against 128 x 128; taken for wide products
// that still fill every SM with them (otherwise the narrower tile keeps more SMs busy).
bool f16x3_use_wide(const TcGemmArgs& g) {
    if (g.N <= 192) return false;
    const int64_t tiles256 = (int64_t)g.batch * ((g.M + BM - 1) / BM) * ((g.N + 255) / 256);
    return tiles256 >= num_sms();
}

namespace {

// ------------------------------------------------------------------ online tuning of the variant
// The factor's FP32-accurate products have three implementations: the FP16 three-product kernel on
// the tile width the heuristic above picks (V_F16), on the other width of {128, 256} (V_F16_ALT,
// for N > 128), and the 3xTF32 kernel with the split done inside the kernel (V_TF32X3: no
// pre-pass launch, half the MMA rate).  With tuning on (slab_autotune(1) or SLAB_AUTOTUNE=1), the
// first calls of each shape class -- log2 buckets of M, N, K and the batch, plus the triangle,
// transposition and shared-operand flags -- run every candidate TUNE_SAMPLES times, timed by an
// event pair on the launching stream, and the class then keeps the candidate with the lowest
// time per flop.  All candidates compute the same product to FP32-level accuracy (the last bits
// differ), so exploring costs nothing but time.  Streams under capture are never timed: they take
// the decided candidate, or V_F16 while a class is still undecided.
enum TuneVariant { V_F16 = 0, V_F16_ALT = 1, V_TF32X3 = 2, NV = 3 };
constexpr int TUNE_SAMPLES = 2;

struct TuneStat {
    double ms_per_gflop[NV] = {0, 0, 0};
    int done[NV] = {0, 0, 0};         // timed samples harvested
    int issued[NV] = {0, 0, 0};       // timed samples launched
    int choice = -1;
};
struct TunePending {
    uint64_t key;
    int v;
    double gflop;
    cudaEvent_t e0, e1;
};
struct Tuner {
    std::mutex mu;
    std::atomic<int> mode{-1};
    std::unordered_map<uint64_t, TuneStat> table;
    std::vector<TunePending> pending;
    std::vector<cudaEvent_t> spare;
};
Tuner& tuner() {
    static Tuner t;
    return t;
}

int tune_mode() {
    Tuner& T = tuner();
    int m = T.mode.load();
    if (m < 0) {
        const char* e = std::getenv("SLAB_AUTOTUNE");
        int want = (e && *e && *e != '0') ? 1 : 0, expect = -1;
        T.mode.compare_exchange_strong(expect, want);
        m = T.mode.load();
    }
    return m;
}

int ceil_log2(int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}
uint64_t tune_key(const TcGemmArgs& g) {
    return (uint64_t)ceil_log2(g.M) | (uint64_t)ceil_log2(g.N) << 6 | (uint64_t)ceil_log2(g.K) << 12 |
           (uint64_t)ceil_log2(g.batch) << 18 | (uint64_t)(g.lower_only != 0) << 24 | (uint64_t)(g.transC != 0) << 25 |
           (uint64_t)f16x3_shared(g) << 26;
}
bool tune_allowed(const TcGemmArgs& g, int v) { return v != V_F16_ALT || g.N > 128; }

// Decide a class once every candidate has its samples: the lowest mean time per flop.
void tune_decide(TuneStat& s, bool alt_ok) {
    int best = -1;
    for (int v = 0; v < NV; ++v) {
        if (v == V_F16_ALT && !alt_ok) continue;
        if (s.done[v] < TUNE_SAMPLES) return;
        if (best < 0 || s.ms_per_gflop[v] / s.done[v] < s.ms_per_gflop[best] / s.done[best]) best = v;
    }
    s.choice = best;
}

// Fold finished timings into the table (caller holds the lock).
void tune_harvest(Tuner& T) {
    for (size_t i = 0; i < T.pending.size();) {
        TunePending& p = T.pending[i];
        const cudaError_t q = cudaEventQuery(p.e1);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        float ms = 0.f;
        if (q == cudaSuccess && cudaEventElapsedTime(&ms, p.e0, p.e1) == cudaSuccess && p.gflop > 0) {
            TuneStat& s = T.table[p.key];
            s.ms_per_gflop[p.v] += ms / p.gflop;
            s.done[p.v] += 1;
            const bool alt_ok = ((p.key >> 6) & 63) > 7;            // N > 128
            if (s.choice < 0) tune_decide(s, alt_ok);
        } else {
            cudaGetLastError();
        }
        T.spare.push_back(p.e0);
        T.spare.push_back(p.e1);
        T.pending[i] = T.pending.back();
        T.pending.pop_back();
    }
}

cudaEvent_t tune_event(Tuner& T) {
    if (!T.spare.empty()) {
        cudaEvent_t e = T.spare.back();
        T.spare.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

slab_status launch_variant(cudaStream_t st, TcGemmArgs& g, unsigned* err, int v) {
    const bool narrow = g.N <= 64;
    if (v == V_TF32X3) {
        g.split = 1;
        return narrow ? launch_tc<64, true>(st, g, err) : launch_tc<128, true>(st, g, err);
    }
    if (narrow) return launch_f16x3<64>(st, g, err);
    const bool wide = f16x3_use_wide(g) != (v == V_F16_ALT && g.N > 128);
    return wide ? launch_f16x3<256>(st, g, err) : launch_f16x3<128>(st, g, err);
}

}  // namespace

// Host entry: validates the layout constraints of the TMA path and launches.
slab_status tc_gemm(cudaStream_t st, TcGemmArgs& g, unsigned* err) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return SLAB_OK;
    if (g.K <= 0 || g.K % BK) return SLAB_EINVAL;
    if (g.ksplit > 1 && (g.K % (g.ksplit * BK) || !g.part || g.lower_only || g.split == 2)) return SLAB_EINVAL;
    if (g.lda % 4 || g.ldb % 4 || g.sA % 4 || g.sB % 4) return SLAB_EINVAL;       // 16-byte strides
    if (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15)) return SLAB_EINVAL;      // 16-byte base
    const bool narrow = g.N <= 64;
    if (g.split == 2) {
        if (g.K % BK16 || !g.w16 || g.w16_bytes < f16x3_work_bytes(g.M, g.N, g.K, g.batch, f16x3_shared(g)) ||
            ((uintptr_t)g.w16 & 255) || g.batch > 65535)
            return SLAB_EINVAL;
        if (tune_mode() == 1) {
            Tuner& T = tuner();
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
            const uint64_t key = tune_key(g);
            int v = V_F16;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            {
                std::lock_guard<std::mutex> lock(T.mu);
                if (!capturing) tune_harvest(T);
                TuneStat& s = T.table[key];
                if (s.choice >= 0) {
                    v = s.choice;
                } else if (!capturing) {
                    int best = -1;                      // the least-sampled candidate still short of samples
                    for (int c = 0; c < NV; ++c)
                        if (tune_allowed(g, c) && s.issued[c] < TUNE_SAMPLES && (best < 0 || s.issued[c] < s.issued[best]))
                            best = c;
                    if (best >= 0) {
                        e0 = tune_event(T);
                        e1 = e0 ? tune_event(T) : nullptr;
                        if (e1) {
                            v = best;
                            s.issued[v] += 1;
                        } else if (e0) {
                            T.spare.push_back(e0);
                            e0 = nullptr;
                        }
                    }
                }
            }
            if (e0) cudaEventRecord(e0, st);
            const slab_status r = launch_variant(st, g, err, v);
            if (e0) {
                cudaEventRecord(e1, st);
                std::lock_guard<std::mutex> lock(T.mu);
                T.pending.push_back(TunePending{key, v, 2e-9 * g.M * g.N * g.K * g.batch, e0, e1});
            }
            return r;
        }
        if (narrow) return launch_f16x3<64>(st, g, err);
        return f16x3_use_wide(g) ? launch_f16x3<256>(st, g, err) : launch_f16x3<128>(st, g, err);
    }
    // few right-hand sides (the solve products): 32-wide tiles leave room for a fifth stage in flight
    if (g.split && g.N <= 32) return launch_tc<32, true>(st, g, err);
    if (g.split) return narrow ? launch_tc<64, true>(st, g, err) : launch_tc<128, true>(st, g, err);
    return narrow ? launch_tc<64, false>(st, g, err) : launch_tc<128, false>(st, g, err);
}

extern "C" int slab_autotune(int mode) {
    Tuner& T = tuner();
    const int prev = tune_mode();
    if (mode == 0 || mode == 1) T.mode.store(mode);
    if (mode == 2) {                                   // forget every decision
        std::lock_guard<std::mutex> lock(T.mu);
        T.table.clear();
    }
    return prev;
}

extern "C" slab_status slab_autotune_stats(int* classes, int* decided, int* tf32x3, int* alt_width) {
    Tuner& T = tuner();
    std::lock_guard<std::mutex> lock(T.mu);
    tune_harvest(T);
    int c = 0, d = 0, t = 0, a = 0;
    for (auto& kv : T.table) {
        ++c;
        if (kv.second.choice >= 0) ++d;
        if (kv.second.choice == V_TF32X3) ++t;
        if (kv.second.choice == V_F16_ALT) ++a;
    }
    if (classes) *classes = c;
    if (decided) *decided = d;
    if (tf32x3) *tf32x3 = t;
    if (alt_width) *alt_width = a;
    return SLAB_OK;
}

size_t f16x3_work_bytes(int64_t M, int64_t N, int64_t K, int batch, bool shared) {
    const size_t b = (size_t)(batch > 0 ? batch : 1);
    size_t w = 2 * align256(b * M * K * 2) + align256(b * M * 4);
    if (!shared) w += 2 * align256(b * N * K * 2) + align256(b * N * 4);
    return w;
}

extern "C" slab_status slab_tc_gemm(int M, int N, int K, float alpha, const float* A, int64_t lda, const float* B,
                                    int64_t ldb, float beta, float* C, int64_t ldc, int trans_c, int split,
                                    unsigned* dev_err, void* stream) {
    if (!A || !B || !C || !dev_err || M < 0 || N < 0) return SLAB_EINVAL;
    TcGemmArgs g;
    g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.transC = trans_c; g.split = split; g.lower_only = 0;
    g.batch = 1; g.sA = g.sB = g.sC = 0;
    g.ksplit = 1; g.part = nullptr;
    g.w16 = nullptr; g.w16_bytes = 0;
    if (split != 2) return tc_gemm((cudaStream_t)stream, g, dev_err);
    // FP16 three-product: scratch for the operand splits from the stream-ordered allocator
    if (K <= 0 || K % 64) return SLAB_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    g.w16_bytes = f16x3_work_bytes(M, N, K, 1, f16x3_shared(g));
    if (cudaMallocAsync(&g.w16, g.w16_bytes, st) != cudaSuccess) {
        cudaGetLastError();
        return SLAB_ENOMEM;
    }
    const slab_status s = tc_gemm(st, g, dev_err);
    if (cudaFreeAsync(g.w16, st) != cudaSuccess) return SLAB_ECUDA;
    return s;
}

// C (FP64, M x N, ldc) += alpha A B^T with A (M x K, lda) and B (N x K, ldb) FP64, FP64-accurate
// on the tensor cores (integer-slice products, above).  K <= 64, K % 32 == 0.  work: float
// slices [OZ_S][M][K] and [OZ_S][N][K] followed by the exponents (M + N ints): ozaki_work_bytes.
size_t ozaki_work_bytes(int64_t M, int64_t N, int K) {
    return (size_t)OZ_S * (M + N) * K * sizeof(float) + (size_t)(M + N) * sizeof(int) + 256;
}

slab_status ozaki_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, int64_t lda,
                       const double* B, int64_t ldb, double* C, int64_t ldc, int lower_only, void* work,
                       unsigned* err) {
    if (M <= 0 || N <= 0) return SLAB_OK;
    if (K <= 0 || K > 64 || K % BK) return SLAB_EINVAL;
    float* As = (float*)work;
    float* Bs = As + (int64_t)OZ_S * M * K;
    int* ea = (int*)(Bs + (int64_t)OZ_S * N * K);
    int* eb = ea + M;
    ozaki_split_kernel<<<(M + 7) / 8, 256, 0, st>>>(A, lda, M, K, As, ea);
    if (cudaGetLastError() != cudaSuccess) return SLAB_ECUDA;
    ozaki_split_kernel<<<(N + 7) / 8, 256, 0, st>>>(B, ldb, N, K, Bs, eb);
    if (cudaGetLastError() != cudaSuccess) return SLAB_ECUDA;
    CUtensorMap ta, tb;
    if (!make_map(&ta, As, M, K, K, OZ_S, (int64_t)M * K, BM)) return SLAB_ECUDA;
    if (!make_map(&tb, Bs, N, K, K, OZ_S, (int64_t)N * K, OZ_BN)) return SLAB_ECUDA;
    static std::atomic<uint32_t> attr_done(0);
    if (!ensure_smem_attr(ozaki_gemm_kernel, OzCfg::SMEM, attr_done)) return SLAB_ECUDA;
    dim3 grid((N + OZ_BN - 1) / OZ_BN, (M + BM - 1) / BM);
    ozaki_gemm_kernel<<<grid, 256, OzCfg::SMEM, st>>>(ta, tb, M, N, K, alpha, ea, eb, C, ldc, lower_only, err);
    return cudaGetLastError() == cudaSuccess ? SLAB_OK : SLAB_ECUDA;
}

extern "C" slab_status slab_fp64_tc_gemm(int M, int N, int K, double alpha, const double* A, int64_t lda,
                                         const double* B, int64_t ldb, double* C, int64_t ldc, void* work,
                                         unsigned* dev_err, void* stream) {
    if (!A || !B || !C || !work || !dev_err || M < 0 || N < 0) return SLAB_EINVAL;
    return ozaki_gemm((cudaStream_t)stream, M, N, K, alpha, A, lda, B, ldb, C, ldc, 0, work, dev_err);
}

extern "C" size_t slab_fp64_tc_gemm_work_bytes(int M, int N, int K) { return ozaki_work_bytes(M, N, K); }
