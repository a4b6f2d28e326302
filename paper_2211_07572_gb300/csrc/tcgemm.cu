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

#include "slab_internal.cuh"

namespace {

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
    static constexpr int STAGES = SPLIT ? 3 : 5;
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
                   int lower_only, int ksplit, float* part, unsigned* err) {
    using Cfg = TcCfg<BN, SPLIT>;
    constexpr int STAGES = Cfg::STAGES;
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    __shared__ uint64_t full_bar[STAGES], conv_bar[STAGES], empty_bar[STAGES], done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    // with ksplit > 1 (single product), blockIdx.z is the K split: K range [zs K/ksplit, (zs+1) K/ksplit)
    const int bn = blockIdx.x, bm = blockIdx.y;
    const int zs = ksplit > 1 ? (int)blockIdx.z : 0;
    const int bz = ksplit > 1 ? 0 : (int)blockIdx.z;
    if (lower_only && bn * BN >= (bm + 1) * BM) return;        // tile strictly above the diagonal
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = K / ksplit / BK;
    const int k0 = zs * nk * BK;
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
            if (ok) mma_commit(&done_bar);
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
        const bool ok = !abort_flag && mbar_wait(&done_bar, 0);
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
                tmem_ld32(tmem + ((uint32_t)(rw * 32) << 16) + (uint32_t)(cc * 32), v);
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
                        float* pb = part + (int64_t)zs * M * N;
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

// C = alpha sum_s part[s] + beta C, part laid out like C (transC: [N][M], else [M][N]), fixed order.
__global__ void splitk_reduce_kernel(int M, int N, int ks, const float* __restrict__ part, float alpha, float beta,
                                     float* C, int64_t ldc, int transC) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)M * N;
    if (e >= tot) return;
    float v = 0.f;
    for (int s = 0; s < ks; ++s) v += part[(int64_t)s * tot + e];
    int64_t idx;
    if (transC) idx = (e / M) * ldc + (e % M);          // e = col * M + row
    else idx = (e / N) * ldc + (e % N);                 // e = row * N + col
    C[idx] = alpha * v + (beta != 0.f ? beta * C[idx] : 0.f);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
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
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(tc_gemm_kernel<BN, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
            return SLAB_ECUDA;
        attr_set = true;
    }
    const int ks = g.ksplit > 1 ? g.ksplit : 1;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, ks > 1 ? ks : g.batch);
    tc_gemm_kernel<BN, SPLIT><<<grid, 256, smem, st>>>(ta, tb, g.M, g.N, g.K, g.alpha, g.beta, g.C, g.ldc, g.sC,
                                                       g.transC, g.lower_only, ks, g.part, err);
    if (cudaGetLastError() != cudaSuccess) return SLAB_ECUDA;
    if (ks > 1) {
        const int64_t tot = (int64_t)g.M * g.N;
        splitk_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g.M, g.N, ks, g.part, g.alpha, g.beta,
                                                                           g.C, g.ldc, g.transC);
        if (cudaGetLastError() != cudaSuccess) return SLAB_ECUDA;
    }
    return SLAB_OK;
}

}  // namespace

// Host entry: validates the layout constraints of the TMA path and launches.
slab_status tc_gemm(cudaStream_t st, const TcGemmArgs& g, unsigned* err) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return SLAB_OK;
    if (g.K <= 0 || g.K % BK) return SLAB_EINVAL;
    if (g.ksplit > 1 && (g.batch != 1 || g.K % (g.ksplit * BK) || !g.part)) return SLAB_EINVAL;
    if (g.lda % 4 || g.ldb % 4 || g.sA % 4 || g.sB % 4) return SLAB_EINVAL;       // 16-byte strides
    if (((uintptr_t)g.A & 15) || ((uintptr_t)g.B & 15)) return SLAB_EINVAL;      // 16-byte base
    const bool narrow = g.N <= 64;
    if (g.split) return narrow ? launch_tc<64, true>(st, g, err) : launch_tc<128, true>(st, g, err);
    return narrow ? launch_tc<64, false>(st, g, err) : launch_tc<128, false>(st, g, err);
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
    return tc_gemm((cudaStream_t)stream, g, dev_err);
}
