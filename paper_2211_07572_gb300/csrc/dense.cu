// Stage 2: factorisation of the block-tridiagonal reduced matrix T
// (Sec. 4, Algorithm 1) and the sweeping solve (Algorithm 2).
//
// T is symmetric positive definite for the SPD kinds, so Algorithm 1's
// S_1 = T_11, S_{j+1} = T_{j+1,j+1} - T_{j+1,j} S_j^{-1} T_{j,j+1} is carried out as a
// block Cholesky: S_j = L_j L_j^T, Y_j = L_j^{-1} T_{j,j+1}, S_{j+1} = T_{j+1,j+1} - Y_j^T Y_j.
//
// Per interface block j the tall matrix W_j = [S_j ; T_{j+1,j} ; I] (3 s_pad x s_pad, the
// middle block absent for the final interface) is eliminated column panel by column panel
// (64 columns): the panel kernel factors the 64 x 64 diagonal tile and multiplies every tile
// below it by L_kk^{-T}; one product C -= A B^T then updates everything right of the panel.
// Rows r of the identity block stay zero in columns < r, so panel kb only touches its first
// (kb+1)*64 rows.  Afterwards the lower blocks of W_j hold Y_j^T and L_j^{-T}, and
// S_{j+1} = T_{j+1,j+1} - Y_j^T (Y_j^T)^T is one more product.  In FP32 every product runs on
// the tensor cores (tcgen05, 3xTF32); the FP64 path uses the same structure on SIMT units.
//
// Algorithm 2 then needs products only (vectors stored right-hand-side major, [k][s_pad]):
//   forward   z_j = L_j^{-1} (f_j - Y_{j-1}^T z_{j-1})
//   backward  u_j = L_j^{-T} (z_j - Y_j u_{j+1}).
#include <algorithm>
#include <cstdio>
#include <vector>

#include "slab_internal.cuh"

namespace {

constexpr int TL = SLAB_TILE;   // 64
constexpr int TLP = TL + 1;
constexpr int PTP = TL + 4;      // row pitch of the panel kernels' tiles: 16-byte rows, rows four banks apart

// C(64x64) += op(A) op(B) over [k0, k1) (multiple of 16); 256 threads, 4x4 per thread.
// op(A)(i,k) = TA ? A[k*lda+i] : A[i*lda+k];  op(B)(k,j) = TB ? B[j*ldb+k] : B[k*ldb+j].
// Columns j >= ncols of B are treated as zero (and not loaded).
template <typename T, bool TA, bool TB>
__device__ inline void tile_gemm(T acc[4][4], const T* __restrict__ A, int64_t lda,
                                 const T* __restrict__ B, int64_t ldb, int k0, int k1, int ncols,
                                 T* sA, T* sB) {
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    for (int kk0 = k0; kk0 < k1; kk0 += 16) {
        __syncthreads();
        for (int idx = tid; idx < 16 * TL; idx += 256) {
            int kk, i;
            if (TA) { kk = idx / TL; i = idx % TL; sA[kk * TLP + i] = A[(int64_t)(kk0 + kk) * lda + i]; }
            else { i = idx / 16; kk = idx % 16; sA[kk * TLP + i] = A[(int64_t)i * lda + kk0 + kk]; }
        }
        for (int idx = tid; idx < 16 * TL; idx += 256) {
            int kk, j;
            if (TB) { j = idx / 16; kk = idx % 16; sB[kk * TLP + j] = j < ncols ? B[(int64_t)j * ldb + kk0 + kk] : T(0); }
            else { kk = idx / TL; j = idx % TL; sB[kk * TLP + j] = j < ncols ? B[(int64_t)(kk0 + kk) * ldb + j] : T(0); }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sA[kk * TLP + ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = sB[kk * TLP + tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
    }
}

// SIMT C = beta C + alpha A B^T (A [M][K], B [N][K] row-major), K multiple of 16.
// transC writes C^T; lower_only skips 64 x 64 output tiles above the diagonal.
template <typename T>
__global__ void __launch_bounds__(256) gemm_tn_kernel(int M, int N, int K, T alpha, const T* A, int64_t lda,
                                                      const T* B, int64_t ldb, T beta, T* C, int64_t ldc,
                                                      int transC, int lower_only, int64_t sA, int64_t sB,
                                                      int64_t sC) {
    __shared__ T sA_[16 * TLP];
    __shared__ T sB_[16 * TLP];
    T* sAm = sA_;
    T* sBm = sB_;
    const int bj = blockIdx.x, bi = blockIdx.y;
    A += (int64_t)blockIdx.z * sA;
    B += (int64_t)blockIdx.z * sB;
    C += (int64_t)blockIdx.z * sC;
    if (lower_only && bj > bi) return;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    const int ncols = min(TL, N - bj * TL);
    tile_gemm<T, false, true>(acc, A + (int64_t)bi * TL * lda, lda, B + (int64_t)bj * TL * ldb, ldb, 0, K, ncols,
                              sAm, sBm);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = bi * TL + ty + 16 * a, c = bj * TL + tx + 16 * b;
            if (r < M && c < N) {
                T* p = transC ? C + (int64_t)c * ldc + r : C + (int64_t)r * ldc + c;
                *p = (beta == T(0) ? T(0) : beta * *p) + alpha * acc[a][b];
            }
        }
}

// SIMT skinny variant (N <= 64) of the same product, K split over gridDim.y CTAs per row tile;
// partial tiles go to ws and the last CTA of a tile (ticket) adds them in split order.
template <typename T>
__global__ void __launch_bounds__(256) gemm_tn_skinny_kernel(int M, int N, int K, T alpha, const T* A,
                                                             int64_t lda, const T* B, int64_t ldb, T beta, T* C,
                                                             int64_t ldc, int transC, T* ws, unsigned* tickets) {
    __shared__ T sA[16 * TLP];
    __shared__ T sB[16 * TLP];
    __shared__ bool last;
    const int bi = blockIdx.x, sp = blockIdx.y, KS = gridDim.y;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int kchunk = K / KS;
    const int k0 = sp * kchunk, k1 = k0 + kchunk;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    tile_gemm<T, false, true>(acc, A + (int64_t)bi * TL * lda, lda, B, ldb, k0, k1, N, sA, sB);
    T* w = ws + ((int64_t)bi * KS + sp) * TL * TL;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) w[(ty + 16 * a) * TL + tx + 16 * b] = acc[a][b];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(tickets + bi, 1u) == (unsigned)(KS - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    const T* w0 = ws + (int64_t)bi * KS * TL * TL;
    for (int e = tid; e < TL * TL; e += 256) {
        const int r = e / TL, c = e % TL;
        T v = T(0);
        for (int q = 0; q < KS; ++q) v += __ldcg(w0 + (int64_t)q * TL * TL + e);
        const int gr = bi * TL + r;
        if (gr < M && c < N) {
            T* p = transC ? C + (int64_t)c * ldc + gr : C + (int64_t)gr * ldc + c;
            *p = (beta == T(0) ? T(0) : beta * *p) + alpha * v;
        }
    }
    if (tid == 0) tickets[bi] = 0;
}

// Cholesky L L^T = S of the 64 x 64 tile S (smem, stride PTP; lower triangle read) and
// Li = L^{-1} (written to smem, stride PTP), by 256 threads in 4 x 4 register blocks, as one sweep
// of right-looking elimination over [S | I] (16 block steps of 4 columns, two barriers each).
// Thread (ti, tj), tj <= ti, holds one block: A_ij while column block tj is not yet eliminated,
// then X_ij, the block of X = L^{-1} under construction (X starts as I).  Block step kt:
//   the diagonal thread factors its 4 x 4 block, L_kk L_kk^T = A_kk, inverts L_kk (reciprocal
//   square roots refined by one Newton step) and continues with X_kk = I;
//   the owners of block column kt publish L_ik = A_ik L_kk^{-T} and continue with X_ik = 0, the
//   owners of block row kt of X apply X_kj := L_kk^{-1} X_kj and publish it;
//   every thread below row kt applies B_ij -= L_ik R_j with R_j = L_jk^T (j > kt, its A block) or
//   R_j = X_kj (j <= kt, its X block).
// L's column block and X's row block share one staging buffer pb[p][4 j + c] (rows of L for
// j > kt, columns of X for j <= kt), so both updates are one product with no divergence, and the
// 16 column owners of a warp read 16 consecutive words per load.  A non-positive or non-finite
// pivot sets SLAB_DEV_NOTSPD and continues with 1.
template <typename T> __device__ __forceinline__ T rsqrt_nr(T a);
template <> __device__ __forceinline__ float rsqrt_nr<float>(float a) {
    float r = rsqrtf(a);
    return r * (1.5f - 0.5f * a * r * r);
}
template <> __device__ __forceinline__ double rsqrt_nr<double>(double a) {
    double r = rsqrt(a);
    return r * (1.5 - 0.5 * a * r * r);
}
// A usable Cholesky pivot: positive and finite (NaN fails both comparisons), in T's own arithmetic.
__device__ __forceinline__ bool pivot_ok(float d) { return d > 0.0f && d <= 3.402823466e38f; }
__device__ __forceinline__ bool pivot_ok(double d) { return d > 0.0 && d <= 1.7976931348623157e308; }

template <typename T>
__device__ __forceinline__ void chol_inv_tile(const T* S, T* Li, unsigned* status) {
    __shared__ T dinv[16];          // L_kk^{-1} (4x4 lower, row-major)
    __shared__ T pb[4 * 64];        // column block kt of L / row block kt of X: [p][4 j + c]
    const int t = threadIdx.x, ti = t >> 4, tj = t & 15;
    T blk[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) blk[r][c] = S[(4 * ti + r) * PTP + 4 * tj + c];
    for (int kt = 0; kt < 16; ++kt) {
        if (ti == kt && tj == kt) {               // 4x4 Cholesky and inverse in registers
            T l[4][4], li[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) { l[r][c] = T(0); li[r][c] = T(0); }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                T d = blk[c][c];
#pragma unroll
                for (int p = 0; p < c; ++p) d -= l[c][p] * l[c][p];
                if (!pivot_ok(d)) { atomicOr(status, SLAB_DEV_NOTSPD); d = T(1); }
                const T rd = rsqrt_nr<T>(d);
                l[c][c] = d * rd;
#pragma unroll
                for (int r = c + 1; r < 4; ++r) {
                    T v = blk[r][c];
#pragma unroll
                    for (int p = 0; p < c; ++p) v -= l[r][p] * l[c][p];
                    l[r][c] = v * rd;
                }
                li[c][c] = rd;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int r = c + 1; r < 4; ++r) {
                    T v = T(0);
#pragma unroll
                    for (int p = c; p < r; ++p) v -= l[r][p] * li[p][c];
                    li[r][c] = v * li[r][r];
                }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    dinv[r * 4 + c] = li[r][c];
                    blk[r][c] = (r == c) ? T(1) : T(0);   // X_kk starts as I
                }
        }
        __syncthreads();
        if (tj == kt && ti > kt) {                // publish L_ik = A_ik L_kk^{-T}; continue with X_ik = 0
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    T v = T(0);
#pragma unroll
                    for (int p = 0; p <= c; ++p) v += blk[r][p] * dinv[c * 4 + p];
                    pb[c * 64 + 4 * ti + r] = v;
                }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) blk[r][c] = T(0);
        }
        if (ti == kt && tj <= kt) {               // X_kt,j = L_kk^{-1} X_kt,j, published
            T o[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    T v = T(0);
#pragma unroll
                    for (int p = 0; p <= r; ++p) v += dinv[r * 4 + p] * blk[p][c];
                    o[r][c] = v;
                }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) { blk[r][c] = o[r][c]; pb[r * 64 + 4 * tj + c] = o[r][c]; }
        }
        __syncthreads();
        if (ti > kt && tj <= ti) {                // B_ij -= L_ik R_j
            T lk[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int p = 0; p < 4; ++p) lk[r][p] = pb[p * 64 + 4 * ti + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                T rj[4];
#pragma unroll
                for (int p = 0; p < 4; ++p) rj[p] = pb[p * 64 + 4 * tj + c];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int p = 0; p < 4; ++p) blk[r][c] -= lk[r][p] * rj[p];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) Li[(4 * ti + r) * PTP + 4 * tj + c] = (tj <= ti) ? blk[r][c] : T(0);
    __syncthreads();
}

// Stage a 64 x 64 tile (row stride ld) in registers, then in shared memory (row stride PTP); 256
// threads.  Every global load of a thread is issued before its first shared store, so a tile costs
// one memory round trip instead of one per element the thread copies.
constexpr int TPT = TL * TL / 256;     // elements of a tile per thread
template <typename T>
__device__ __forceinline__ void tile_fetch(const T* src, int64_t ld, T (&v)[TPT]) {
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int i = threadIdx.x + 256 * q;
        v[q] = src[(int64_t)(i / TL) * ld + i % TL];
    }
}
template <typename T>
__device__ __forceinline__ void tile_stash(const T (&v)[TPT], T* dst) {
#pragma unroll
    for (int q = 0; q < TPT; ++q) {
        const int i = threadIdx.x + 256 * q;
        dst[(i / TL) * PTP + i % TL] = v[q];
    }
}

// Four consecutive shared-memory values, 16-byte aligned: one 128-bit load (float), two (double).
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// acc[a][b] += sum_l X[ty + 16 a][l] Y[tx + 16 b][l] for 64 x 64 tiles X, Y in shared memory (row
// pitch PTP, 16-byte aligned), four l at a time: eight vector loads per 64 FMAs; the 16 rows
// tx + 16 b of a warp's loads are PTP = 68 words apart, so a phase of eight lanes hits eight
// distinct bank quads.
template <typename T>
__device__ __forceinline__ void tile_nt(const T* X, const T* Y, T acc[4][4], int ty, int tx) {
#pragma unroll 4
    for (int l = 0; l < TL; l += 4) {
        T av[4][4], bv[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a) ld4(X + (ty + 16 * a) * PTP + l, av[a]);
#pragma unroll
        for (int b = 0; b < 4; ++b) ld4(Y + (tx + 16 * b) * PTP + l, bv[b]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a][u] * bv[b][u];
    }
}

// Panel of tile column kb of the tall matrix Wt (leading dimension ld), in two launches.
// panel_diag_kernel (one CTA per matrix of the batch): Cholesky of the diagonal tile
// Wt[kb][kb] = L L^T and Linv = L^{-1} to Lw (64 x 64 per matrix, row-major).
template <typename T>
__global__ void __launch_bounds__(256) panel_diag_kernel(const T* Wt, int64_t ld, int kb, unsigned* status,
                                                         int64_t bstride, T* Lw) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    T* Li = S + TL * PTP;
    const int tid = threadIdx.x;
    Wt += (int64_t)blockIdx.y * bstride;
    const T* D = Wt + (int64_t)kb * TL * ld + (int64_t)kb * TL;
    {
        T v[TPT];
        tile_fetch<T>(D, ld, v);
        tile_stash<T>(v, S);
    }
    __syncthreads();
    chol_inv_tile<T>(S, Li, status);
    T* out = Lw + (int64_t)blockIdx.y * TL * TL;
    for (int i = tid; i < TL * TL; i += 256) out[i] = Li[(i / TL) * PTP + i % TL];
}

// panel_apply_kernel: CTA x replaces the tile Wt[kb+1+x][kb] by itself times L^{-T}.  DIAG: every
// CTA factors the diagonal tile itself (the same arithmetic as panel_diag_kernel, so every CTA
// obtains the same L^{-1}) instead of reading Lw -- one launch per panel where the row tiles of the
// batch fit in one wave, so the redundant 64 x 64 factorisations cost no extra time.
template <typename T, bool DIAG>
__global__ void __launch_bounds__(256) panel_apply_kernel(T* Wt, int64_t ld, int kb, int64_t bstride,
                                                          const T* Lw, unsigned* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Li = reinterpret_cast<T*>(smem_raw);
    T* X = Li + TL * PTP;
    T* S = X + TL * PTP;                          // DIAG only: the diagonal tile
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int r = kb + 1 + blockIdx.x;
    Wt += (int64_t)blockIdx.y * bstride;
    T* src = Wt + (int64_t)r * TL * ld + (int64_t)kb * TL;
    {
        T vl[TPT], vx[TPT];
        if (DIAG) tile_fetch<T>(Wt + (int64_t)kb * TL * ld + (int64_t)kb * TL, ld, vl);
        else tile_fetch<T>(Lw + (int64_t)blockIdx.y * TL * TL, TL, vl);
        tile_fetch<T>(src, ld, vx);
        tile_stash<T>(vl, DIAG ? S : Li);
        tile_stash<T>(vx, X);
    }
    __syncthreads();
    if (DIAG) chol_inv_tile<T>(S, Li, status);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    tile_nt<T>(X, Li, acc, ty, tx);       // out = X Li^T
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) src[(int64_t)(ty + 16 * a) * ld + tx + 16 * b] = acc[a][b];
}

// Two panels kb, kb+1 of the tall Cholesky in one launch after panel_diag_kernel(kb): CTA x owns
// row tile r = kb+1+x and
//   scales its tile of panel kb, P_r = W[r][kb] L^{-T} (written back, except for r = kb+1),
//   recomputes P_{kb+1} = W[kb+1][kb] L^{-T} from the unscaled tile (every CTA reads it; its scaled
//   value is used only here, so it is never written),
//   applies panel kb to panel kb+1: W[r][kb+1] -= P_r P_{kb+1}^T,
// and the CTA of r = kb+1 then factors the updated diagonal tile of panel kb+1 (Cholesky and
// inverse, as panel_diag_kernel) into Lw2.  Panel kb+1 is finished by panel_apply_kernel(kb+1, Lw2).
// DIAG: every CTA factors panel kb's diagonal tile itself, as panel_apply_kernel<T, true>.
template <typename T, bool DIAG>
__global__ void __launch_bounds__(256) panel_pair_kernel(T* Wt, int64_t ld, int kb, int64_t bstride, const T* Lw,
                                                         T* Lw2, unsigned* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Li = reinterpret_cast<T*>(smem_raw);
    T* X = Li + TL * PTP;
    T* Y = X + TL * PTP;
    T* C = Y + TL * PTP;
    T* S = C + TL * PTP;                          // DIAG only: panel kb's diagonal tile
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int r = kb + 1 + blockIdx.x;
    Wt += (int64_t)blockIdx.y * bstride;
    T* src = Wt + (int64_t)r * TL * ld + (int64_t)kb * TL;
    const T* src1 = Wt + (int64_t)(kb + 1) * TL * ld + (int64_t)kb * TL;
    T* dst = Wt + (int64_t)r * TL * ld + (int64_t)(kb + 1) * TL;
    {
        T vl[TPT], vx[TPT], vy[TPT], vc[TPT];
        if (DIAG) tile_fetch<T>(Wt + (int64_t)kb * TL * ld + (int64_t)kb * TL, ld, vl);
        else tile_fetch<T>(Lw + (int64_t)blockIdx.y * TL * TL, TL, vl);
        tile_fetch<T>(src, ld, vx);
        tile_fetch<T>(src1, ld, vy);
        tile_fetch<T>(dst, ld, vc);
        tile_stash<T>(vl, DIAG ? S : Li);
        tile_stash<T>(vx, X);
        tile_stash<T>(vy, Y);
        tile_stash<T>(vc, C);
    }
    __syncthreads();
    if (DIAG) chol_inv_tile<T>(S, Li, status);
    T p[4][4], q[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[a][b] = q[a][b] = T(0);
    tile_nt<T>(X, Li, p, ty, tx);                  // P_r
    tile_nt<T>(Y, Li, q, ty, tx);                  // P_{kb+1}
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            X[(ty + 16 * a) * PTP + tx + 16 * b] = p[a][b];
            Y[(ty + 16 * a) * PTP + tx + 16 * b] = q[a][b];
            if (r != kb + 1) src[(int64_t)(ty + 16 * a) * ld + tx + 16 * b] = p[a][b];
        }
    __syncthreads();
    T u[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) u[a][b] = C[(ty + 16 * a) * PTP + tx + 16 * b];
    {
        T pq[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) pq[a][b] = T(0);
        tile_nt<T>(X, Y, pq, ty, tx);              // P_r P_{kb+1}^T
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) u[a][b] -= pq[a][b];
    }
    if (r != kb + 1) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) dst[(int64_t)(ty + 16 * a) * ld + tx + 16 * b] = u[a][b];
        return;
    }
    __syncthreads();                               // (uniform: this CTA alone) all reads of C done
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) C[(ty + 16 * a) * PTP + tx + 16 * b] = u[a][b];
    __syncthreads();
    chol_inv_tile<T>(C, X, status);                // X := L^{-1} of panel kb+1's diagonal tile
    T* out = Lw2 + (int64_t)blockIdx.y * TL * TL;
    for (int i = tid; i < TL * TL; i += 256) out[i] = X[(i / TL) * PTP + i % TL];
}

// Panels kb and kb+1 complete in one launch (every CTA factors both diagonal tiles itself): CTA x
// owns row tile r = kb+1+x, x = 0 .. nrt (one more than panel kb's row tiles: with the identity
// block starting on a tile boundary, the last one enters with panel kb+1, and its tile of panel kb
// is zero), and
//   factors W[kb][kb] = L L^T,  P_r = W[r][kb] L^{-T} (written back, except for r = kb+1),
//   P_{kb+1} = W[kb+1][kb] L^{-T} (recomputed from the unscaled tile, never written),
//   W[r][kb+1] -= P_r P_{kb+1}^T and the updated diagonal tile D = W[kb+1][kb+1] - P_{kb+1} P_{kb+1}^T,
//   factors D = L' L'^T and writes W[r][kb+1] L'^{-T} (except for r = kb+1, the diagonal tile).
// The same arithmetic in every CTA gives every CTA the same L^{-1} and L'^{-1}.
template <typename T>
__global__ void __launch_bounds__(256) panel_pair_full_kernel(T* Wt, int64_t ld, int kb, int64_t bstride,
                                                              unsigned* status) {
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Li = reinterpret_cast<T*>(smem_raw);
    T* X = Li + TL * PTP;
    T* Y = X + TL * PTP;
    T* C = Y + TL * PTP;
    T* S = C + TL * PTP;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int r = kb + 1 + blockIdx.x;
    Wt += (int64_t)blockIdx.y * bstride;
    T* src = Wt + (int64_t)r * TL * ld + (int64_t)kb * TL;
    const T* src1 = Wt + (int64_t)(kb + 1) * TL * ld + (int64_t)kb * TL;
    T* dst = Wt + (int64_t)r * TL * ld + (int64_t)(kb + 1) * TL;
    T vd[TPT];
    {
        T vs[TPT], vx[TPT], vy[TPT], vc[TPT];
        tile_fetch<T>(Wt + (int64_t)kb * TL * ld + (int64_t)kb * TL, ld, vs);
        tile_fetch<T>(src, ld, vx);
        tile_fetch<T>(src1, ld, vy);
        tile_fetch<T>(dst, ld, vc);
        tile_fetch<T>(Wt + (int64_t)(kb + 1) * TL * ld + (int64_t)(kb + 1) * TL, ld, vd);
        tile_stash<T>(vs, S);
        tile_stash<T>(vx, X);
        tile_stash<T>(vy, Y);
        tile_stash<T>(vc, C);
    }
    __syncthreads();
    chol_inv_tile<T>(S, Li, status);               // ends with a barrier: S is free
    tile_stash<T>(vd, S);
    T p[4][4], q[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[a][b] = q[a][b] = T(0);
    tile_nt<T>(X, Li, p, ty, tx);                  // P_r
    tile_nt<T>(Y, Li, q, ty, tx);                  // P_{kb+1}
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            X[(ty + 16 * a) * PTP + tx + 16 * b] = p[a][b];
            Y[(ty + 16 * a) * PTP + tx + 16 * b] = q[a][b];
            if (r != kb + 1) src[(int64_t)(ty + 16 * a) * ld + tx + 16 * b] = p[a][b];
        }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[a][b] = q[a][b] = T(0);
    tile_nt<T>(X, Y, p, ty, tx);                   // P_r P_{kb+1}^T
    tile_nt<T>(Y, Y, q, ty, tx);                   // P_{kb+1} P_{kb+1}^T
    T u[4][4], d[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            u[a][b] = C[(ty + 16 * a) * PTP + tx + 16 * b] - p[a][b];
            d[a][b] = S[(ty + 16 * a) * PTP + tx + 16 * b] - q[a][b];
        }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            C[(ty + 16 * a) * PTP + tx + 16 * b] = u[a][b];
            S[(ty + 16 * a) * PTP + tx + 16 * b] = d[a][b];
        }
    __syncthreads();
    chol_inv_tile<T>(S, Li, status);               // L'^{-1}
    if (r == kb + 1) return;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[a][b] = T(0);
    tile_nt<T>(C, Li, p, ty, tx);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dst[(int64_t)(ty + 16 * a) * ld + tx + 16 * b] = p[a][b];
}

// Ones on the diagonal of the s_pad x s_pad block B (blockIdx.y selects one of a batch, stride apart);
// the zeros come from a memset before it.
template <typename T>
__global__ void set_diagonal_kernel(T* B, int s_pad, int64_t stride) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < s_pad) B[(int64_t)blockIdx.y * stride + (int64_t)i * (s_pad + 1)] = T(1);
}

// B = I for nb blocks of s_pad x s_pad, stride elements apart: a memset of each block (full
// bandwidth) and one launch for the diagonals.
template <typename T>
slab_status set_identity(slab_handle* h, T* B, int s_pad, int64_t stride, int nb) {
    const int64_t blk = (int64_t)s_pad * s_pad;
    if (stride == blk) SLAB_CK(h, cudaMemsetAsync(B, 0, (size_t)nb * blk * sizeof(T), h->stream));
    else
        for (int i = 0; i < nb; ++i) SLAB_CK(h, cudaMemsetAsync(B + i * stride, 0, blk * sizeof(T), h->stream));
    set_diagonal_kernel<T><<<dim3((unsigned)((s_pad + 255) / 256), nb), 256, 0, h->stream>>>(B, s_pad, stride);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

// out[c][r] = in[r][c] for the 64 x 64 tile (blockIdx.y, blockIdx.x) of a rows x cols block, 256
// threads: every thread issues its 16 loads (rows of in, coalesced) before its first shared store,
// then writes 16 elements (rows of out, coalesced).  tile[.][65]: column reads are conflict-free.
template <typename T>
__device__ __forceinline__ void transpose_tile64(const T* __restrict__ in, int64_t ldin, T* __restrict__ out,
                                                 int64_t ldout, int rows, int cols) {
    __shared__ T tile[64][65];
    const int c0 = blockIdx.x * 64, r0 = blockIdx.y * 64;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    T v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int r = r0 + ty + 4 * q, c = c0 + tx;
        v[q] = (r < rows && c < cols) ? in[(int64_t)r * ldin + c] : T(0);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) tile[ty + 4 * q][tx] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const int c = c0 + ty + 4 * q, r = r0 + tx;
        if (r < rows && c < cols) out[(int64_t)c * ldout + r] = tile[tx][ty + 4 * q];
    }
}

// out = in^T for an n x n block (both row-major, leading dimension n); blockIdx.z selects one of a
// batch of blocks sin / sout elements apart.
template <typename T>
__global__ void __launch_bounds__(256) transpose_kernel(const T* __restrict__ in, T* __restrict__ out, int n,
                                                        int64_t sin, int64_t sout) {
    transpose_tile64<T>(in + (int64_t)blockIdx.z * sin, n, out + (int64_t)blockIdx.z * sout, n, n, n);
}

template <typename T>
slab_status transpose_batched(slab_handle* h, const T* in, int64_t sin, T* out, int64_t sout, int n, int batch) {
    if (batch <= 0) return SLAB_OK;
    dim3 grid((n + 63) / 64, (n + 63) / 64, batch);
    SLAB_PROF(h, KC_OTHER);
    transpose_kernel<T><<<grid, 256, 0, h->stream>>>(in, out, n, sin, sout);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T>
slab_status transpose(slab_handle* h, const T* in, T* out, int n) {
    return transpose_batched<T>(h, in, 0, out, 0, n, 1);
}

// The factor's Schur, trailing and (3-D) T-assembly products (FP32, 3xTF32 accuracy requested)
// run as three FP16 products of row-scaled hi/lo splits when the handle holds a large enough
// work buffer (it exists only while the factor runs).
inline bool use_f16x3(slab_handle* h, int cls, TcGemmArgs& g) {
    if (!h->w16 || g.split != 1 || (cls != KC_SYRK && cls != KC_TRAIL && cls != KC_ASSEMBLE) || g.K % 64)
        return false;
    if (f16x3_work_bytes(g.M, g.N, g.K, g.batch, f16x3_shared(g)) > h->w16_bytes) return false;
    g.split = 2;
    g.w16 = h->w16;
    g.w16_bytes = h->w16_bytes;
    return true;
}

// FP32 C = beta C + alpha A B^T for N <= NB right-hand sides (the single-load solves' products): the product
// streams A once.  A block owns 32 rows (a warp four of them); per 128-wide K chunk the block stages
// the N x 128 slice of B in shared memory once (so B is read once per block, not once per warp), and
// every lane multiplies its float4 of the four rows with it, the next chunk of A already loaded
// into registers.  Exact FP32 FMAs; one warp reduction per output at the end.  blockIdx.y is the
// batch index (sA, sB, sC element strides).  Needs K, lda and ldb multiples of 4 and 16-byte
// aligned A and B.
constexpr int SK_ROWS = 32;                          // rows per block (four per warp)
template <int NB>
__global__ void __launch_bounds__(256, 2) skinny_nt_kernel(int M, int N, int K, float alpha, const float* __restrict__ A,
                                                           int64_t lda, int64_t sA, const float* __restrict__ B,
                                                           int64_t ldb, int64_t sB, float beta, float* C, int64_t ldc,
                                                           int64_t sC, int transC) {
    __shared__ float4 bs[NB][32];                     // B[n][k0 .. k0 + 127]
    __shared__ float red[8][4 * NB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row0 = (blockIdx.x * 8 + warp) * 4;
    A += (int64_t)blockIdx.y * sA;
    B += (int64_t)blockIdx.y * sB;
    C += (int64_t)blockIdx.y * sC;
    float acc[4][NB];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int n = 0; n < NB; ++n) acc[r][n] = 0.f;
    const float* ar[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) ar[r] = A + (int64_t)min(row0 + r, M - 1) * lda;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
        a[r] = (4 * lane < K) ? __ldg(reinterpret_cast<const float4*>(ar[r] + 4 * lane)) : zero;
    for (int k0 = 0; k0 < K; k0 += 128) {
        __syncthreads();                              // the previous chunk of bs is consumed
        for (int e = threadIdx.x; e < NB * 32; e += 256) {
            const int n = e >> 5, kk = k0 + 4 * (e & 31);
            bs[n][e & 31] = (n < N && kk < K) ? __ldg(reinterpret_cast<const float4*>(B + (int64_t)n * ldb + kk)) : zero;
        }
        __syncthreads();
        float4 an[4];                                 // next chunk of A
        const int kn = k0 + 128 + 4 * lane;
#pragma unroll
        for (int r = 0; r < 4; ++r) an[r] = (kn < K) ? __ldg(reinterpret_cast<const float4*>(ar[r] + kn)) : zero;
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            const float4 b = bs[n][lane];
#pragma unroll
            for (int r = 0; r < 4; ++r)
                acc[r][n] = fmaf(a[r].x, b.x, fmaf(a[r].y, b.y, fmaf(a[r].z, b.z, fmaf(a[r].w, b.w, acc[r][n]))));
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = an[r];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int n = 0; n < NB; ++n) {
            float v = acc[r][n];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][r * NB + n] = v;
        }
    __syncwarp();
    // lane j writes output j, j + 32, ... of the warp's 4 x N block
    for (int e = lane; e < 4 * N; e += 32) {
        const int r = e / N, n = e % N, row = row0 + r;
        if (row < M) {
            float* c = transC ? C + (int64_t)n * ldc + row : C + (int64_t)row * ldc + n;
            *c = (beta == 0.f ? 0.f : beta * *c) + alpha * red[warp][r * NB + n];
        }
    }
}

// The skinny kernel serves a product when N is small and the layout allows 16-byte loads.
inline bool skinny_ok(int N, int K, const float* A, int64_t lda, int64_t sA, const float* B, int64_t ldb,
                      int64_t sB, int lower_only) {
    // N <= 4 (single loads, as in the batched problems): the tensor-core path would pad N to 64.  From
    // 5 to 16 loads the 3xTF32 tensor-core kernel streams A at least as fast (measured on GB300).
    return N >= 1 && N <= 4 && !lower_only && K % 4 == 0 && lda % 4 == 0 && ldb % 4 == 0 && sA % 4 == 0 &&
           sB % 4 == 0 && ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0;
}

slab_status launch_skinny(slab_handle* h, int M, int N, int K, float alpha, const float* A, int64_t lda, int64_t sA,
                          const float* B, int64_t ldb, int64_t sB, float beta, float* C, int64_t ldc, int64_t sC,
                          int transC, int batch) {
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        dim3 grid((unsigned)((M + SK_ROWS - 1) / SK_ROWS), (unsigned)nb);
        const float* Ab = A + (int64_t)b0 * sA;
        const float* Bb = B + (int64_t)b0 * sB;
        float* Cb = C + (int64_t)b0 * sC;
        skinny_nt_kernel<4><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, Ab, lda, sA, Bb, ldb, sB, beta, Cb, ldc, sC,
                                                         transC);
        SLAB_CK_LAUNCH(h);
    }
    return SLAB_OK;
}

// C = beta C + alpha A B^T on the unit of this precision: tensor cores for FP32, SIMT for FP64.
template <typename T>
slab_status gemm_tn(slab_handle* h, int cls, int M, int N, int K, T alpha, const T* A, int64_t lda, const T* B,
                    int64_t ldb, T beta, T* C, int64_t ldc, int transC, int lower_only, int triA = 0);

template <>
slab_status gemm_tn<float>(slab_handle* h, int cls, int M, int N, int K, float alpha, const float* A, int64_t lda,
                           const float* B, int64_t ldb, float beta, float* C, int64_t ldc, int transC,
                           int lower_only, int triA) {
    SLAB_PROF(h, cls);
    if (skinny_ok(N, K, A, lda, 0, B, ldb, 0, lower_only))
        return launch_skinny(h, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, transC, 1);
    TcGemmArgs g;
    g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.transC = transC; g.split = h->tf32_now ? 0 : 1; g.lower_only = lower_only;
    g.batch = 1; g.sA = g.sB = g.sC = 0;
    g.ksplit = 1; g.part = nullptr;
    g.w16 = nullptr; g.w16_bytes = 0;
    g.triA = triA;
    if (use_f16x3(h, cls, g)) {
        // FP16 three-product path (factor products)
    } else if (N <= 64 && !lower_only && h->wPart) {     // skinny: split K over CTAs
        const int64_t cap = (int64_t)splitk_part_bytes(h->td.s_pad) / sizeof(float);
        int ks = 1;
        while (2 * ks <= SLAB_SPLITK && (M + 127) / 128 * ks < 148 && K % (2 * ks * 32) == 0 &&
               (int64_t)2 * ks * M * N <= cap)
            ks *= 2;
        g.ksplit = ks;
        g.part = (float*)h->wPart;
    }
    const slab_status st = tc_gemm(h->stream, g, h->dstatus);
    if (st == SLAB_ECUDA && h->err == SLAB_OK) h->err = SLAB_ECUDA;
    prof_extra(h, cls, tc_gemm_extra_launches(g));
    return st;
}

template <typename T>
__global__ void scale_matrix_kernel(T* C, int64_t ldc, int M, int N, T beta) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    T* p = C + (e / N) * ldc + e % N;
    *p = beta == T(0) ? T(0) : beta * *p;
}

// C = beta C + alpha A B^T for N <= 8 (right-hand sides): one warp per row of A, lanes over K
// (coalesced), so the product streams A once at memory speed.
template <typename T, int NB>
__global__ void __launch_bounds__(256) gemv_rows_kernel(int M, int N, int K, T alpha, const T* __restrict__ A,
                                                        int64_t lda, const T* __restrict__ B, int64_t ldb, T beta,
                                                        T* C, int64_t ldc, int transC) {
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= M) return;
    T acc[NB];
#pragma unroll
    for (int r = 0; r < NB; ++r) acc[r] = T(0);
    const T* a = A + (int64_t)row * lda;
    for (int k = lane; k < K; k += 32) {
        const T av = a[k];
#pragma unroll
        for (int r = 0; r < NB; ++r)
            if (r < N) acc[r] += av * B[(int64_t)r * ldb + k];
    }
#pragma unroll
    for (int r = 0; r < NB; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int r = 0; r < NB; ++r) {
            if (r >= N) break;
            T* c = transC ? C + (int64_t)r * ldc + row : C + (int64_t)row * ldc + r;
            *c = (beta == T(0) ? T(0) : beta * *c) + alpha * acc[r];
        }
    }
}

template <>
slab_status gemm_tn<double>(slab_handle* h, int cls, int M, int N, int K, double alpha, const double* A,
                            int64_t lda, const double* B, int64_t ldb, double beta, double* C, int64_t ldc,
                            int transC, int lower_only, int /*triA: the FP64 products read all of A*/) {
    if (N <= 8 && !lower_only && M > 0) {
        SLAB_PROF(h, cls);
        gemv_rows_kernel<double, 8><<<(M + 7) / 8, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                                       transC);
        SLAB_CK_LAUNCH(h);
        return SLAB_OK;
    }
    if (h->fp64tc_now && !transC && K % 32 == 0 && M > 0 && N > 0) {
        // FP64-accurate tensor-core product, K in chunks of 64
        SLAB_PROF(h, cls);
        if (beta != 1.0) {
            scale_matrix_kernel<double><<<(unsigned)(((int64_t)M * N + 255) / 256), 256, 0, h->stream>>>(C, ldc, M, N,
                                                                                                         beta);
            SLAB_CK_LAUNCH(h);
        }
        for (int k0 = 0; k0 < K; k0 += 64) {
            const int kc = std::min(64, K - k0);
            const slab_status st = ozaki_gemm(h->stream, M, N, kc, alpha, A + k0, lda, B + k0, ldb, C, ldc, lower_only,
                                              h->ozw, h->dstatus);
            if (st) {
                if (h->err == SLAB_OK) h->err = st;
                return st;
            }
        }
        // launches beyond the one counted: the scaling of C and three per K chunk (two splits, product)
        prof_extra(h, cls, (beta != 1.0 ? 1 : 0) + 3 * ((K + 63) / 64) - 1);
        return SLAB_OK;
    }
    SLAB_PROF(h, cls);
    if (N <= 64 && !lower_only && h->wTickets) {
        int KS = K / 256;
        if (KS < 1) KS = 1;
        if (KS > SLAB_SPLITK) KS = SLAB_SPLITK;
        while (K % (KS * 16)) --KS;
        dim3 grid((M + TL - 1) / TL, KS);
        gemm_tn_skinny_kernel<double><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                                   transC, (double*)h->wPart, h->wTickets);
    } else {
        dim3 grid((N + TL - 1) / TL, (M + TL - 1) / TL);
        gemm_tn_kernel<double><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, transC,
                                                            lower_only, 0, 0, 0);
    }
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

// ---------------------------------------------------------------- indefinite kind (Helmholtz)
// Blocked Gauss-Jordan elimination of the augmented system of interface j
//   top    Gt = [ S_j        | T_{j,j+1}    | I ]      (s_pad x wt, wt = 3 s_pad; 2 s_pad for the last j)
//   bottom Gb = [ T_{j+1,j}  | T_{j+1,j+1}      ]      (s_pad x 2 s_pad)
// eliminating the S_j columns in panels of 64.  At the end the top rows hold (in pivot order)
// [I | S_j^{-1} T_{j,j+1} | S_j^{-1}] and the bottom right block is S_{j+1} of Algorithm 1.
// Rows are never swapped: perm[c] records the physical top row that pivots on column c.
// Pivot rows of a panel are chosen by tournament pivoting: warps run partial-pivoting
// elimination on 128-row groups of the not-yet-pivoted rows, keep 64 winners each, and winners
// are merged pairwise (original row values) up to one set of 64.  The panel step is then
//   A11 = G[piv, panel],  X = A11^{-1} G[piv, rest],  G[piv, rest] = X,
//   G[other, rest] -= G[other, panel] X       (tensor-core rank-64 update).
constexpr int GJ_LEAF = 128;          // rows per tournament group
constexpr int GJ_WARPS = 2;           // tournament warps per CTA

struct GjWork {
    int* act;         // [2][s_pad] not-yet-pivoted top rows, double-buffered by panel parity
    int* perm;        // [s_pad] physical row pivoting on column c
    int* pflag;       // [s_pad] panel index + 1 at which the row pivoted (0: not yet)
    int* cand;        // tournament winner sets, [nodes][64]
    unsigned* tick;   // tournament tickets, [nodes]
    int* piv;         // [64] pivot rows of the current panel
};

__host__ __device__ inline int gj_level_count(int L, int l) {          // nodes at tournament level l
    int c = L;
    for (int i = 0; i < l; ++i) c = (c + 1) / 2;
    return c;
}
__host__ __device__ inline int gj_level_off(int L, int l) {
    int o = 0, c = L;
    for (int i = 0; i < l; ++i) { o += c; c = (c + 1) / 2; }
    return o;
}
__host__ __device__ inline int gj_nodes(int L) {                       // all nodes, leaves to root
    int o = 0, c = L;
    while (c > 1) { o += c; c = (c + 1) / 2; }
    return o + 1;
}

// Partial-pivoting elimination by one warp on nr (64..128) rows x 64 columns held in A (stride 65);
// rows[] are the physical G rows of A's rows.  Writes the 64 chosen physical rows, in order, to out.
template <typename T>
__device__ void gj_warp_gepp(T* A, const int* rows, int nr, int* out) {
    const int lane = threadIdx.x & 31;
    bool chosen[4] = {false, false, false, false};
    for (int j = 0; j < 64; ++j) {
        T best = T(-1);
        int bi = 1 << 30;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int r = lane + 32 * q;
            if (r < nr && !chosen[q]) {
                T v = fabs(A[r * 65 + j]);
                if (v != v) v = T(INFINITY);                  // a NaN is picked, and flagged at A11^{-1}
                if (v > best) { best = v; bi = r; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (bi >= nr) bi = 0;                             // not reached: nr >= 64 unchosen candidates
        if ((bi & 31) == lane) chosen[bi >> 5] = true;
        if (lane == 0) out[j] = rows[bi];
        const T pv = A[bi * 65 + j];
        if (best > T(0)) {
            // the pivot row in registers, the update unrolled over compile-time columns (in blocks of
            // 8 skipped while left of j): the loads of a row are independent of its stores, so they
            // pipeline instead of alternating load -> FMA -> store one column at a time
            T prow[64];
#pragma unroll
            for (int c = 0; c < 64; ++c) prow[c] = A[bi * 65 + c];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = lane + 32 * q;
                if (r < nr && !chosen[q]) {
                    T* Ar = A + r * 65;
                    const T l = Ar[j] / pv;
#pragma unroll
                    for (int cb = 0; cb < 8; ++cb) {
                        if (8 * cb + 7 > j) {
#pragma unroll
                            for (int cc = 0; cc < 8; ++cc) {
                                const int c = 8 * cb + cc;
                                if (c > j) Ar[c] -= l * prow[c];
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
    }
}

// One launch per panel: leaves, pairwise merges (ticketed, deterministic), and at the root the
// panel's pivot rows, their flags and perm entries, and the compacted list of remaining rows.
template <typename T>
// (pivot selection runs in FP32 whatever the storage type: it only chooses rows, the elimination
// itself is done in T by the kernels below)
__global__ void __launch_bounds__(32 * GJ_WARPS) gj_tournament_kernel(const T* __restrict__ G, int64_t ld,
                                                                       int c0, int panel, int nact, GjWork w,
                                                                       const int* act, int* act_next) {
    extern __shared__ unsigned char gj_smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* A = reinterpret_cast<float*>(gj_smem) + (size_t)wid * GJ_LEAF * 65;
    __shared__ int rows_s[GJ_WARPS][GJ_LEAF];
    int* rows = rows_s[wid];
    const int L = (nact + GJ_LEAF - 1) / GJ_LEAF;
    int node = blockIdx.x * GJ_WARPS + wid;
    if (node >= L) return;
    int lvl = 0;
    int nr = min(GJ_LEAF, nact - node * GJ_LEAF);
    for (int i = lane; i < nr; i += 32) rows[i] = act[node * GJ_LEAF + i];
    while (true) {
        __syncwarp();
        // 16 loads in flight per lane (rows are scattered over G, each 64-column row segment coalesced)
        for (int i0 = 0; i0 < nr * 64; i0 += 32 * 16) {
            T v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int idx = i0 + u * 32 + lane;
                v[u] = idx < nr * 64 ? G[(int64_t)rows[idx >> 6] * ld + c0 + (idx & 63)] : T(0);
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int idx = i0 + u * 32 + lane;
                if (idx < nr * 64) A[(idx >> 6) * 65 + (idx & 63)] = (float)v[u];
            }
        }
        __syncwarp();
        int* out = w.cand + (gj_level_off(L, lvl) + node) * 64;
        gj_warp_gepp<float>(A, rows, nr, out);
        __syncwarp();
        if (gj_level_count(L, lvl) == 1) break;         // root
        const int parent = node >> 1;
        const int nchild = ((node ^ 1) < gj_level_count(L, lvl)) ? 2 : 1;
        __threadfence();
        unsigned tk = 0;
        if (lane == 0) tk = atomicAdd(w.tick + gj_level_off(L, lvl + 1) + parent, 1u);
        tk = __shfl_sync(0xffffffffu, tk, 0);
        if ((int)tk + 1 < nchild) return;               // the sibling finishes the merge
        __threadfence();
        const int* c0p = w.cand + (gj_level_off(L, lvl) + 2 * parent) * 64;
        nr = nchild * 64;
        for (int i = lane; i < nr; i += 32) rows[i] = __ldcg(c0p + i);
        node = parent;
        ++lvl;
    }
    // root: the panel's pivot rows
    const int* win = w.cand + (gj_level_off(L, lvl) + node) * 64;
    for (int i = lane; i < 64; i += 32) {
        const int r = __ldcg(win + i);
        w.piv[i] = r;
        w.perm[c0 + i] = r;
        w.pflag[r] = panel + 1;
    }
    __syncwarp();
    __threadfence();
    // every other warp has taken its ticket: reset them for the next panel
    for (int i = lane; i < gj_nodes(L); i += 32) w.tick[i] = 0u;
    // remaining rows, in order: 8 groups of 32 per round, their loads issued before the ballots
    int base = 0;
    for (int i0 = 0; i0 < nact; i0 += 32 * 8) {
        int r[8];
        bool keep[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + 32 * u + lane;
            r[u] = i < nact ? act[i] : -1;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) keep[u] = r[u] >= 0 && __ldcg(w.pflag + r[u]) != panel + 1;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const unsigned bal = __ballot_sync(0xffffffffu, keep[u]);
            if (keep[u]) act_next[base + __popc(bal & ((1u << lane) - 1u))] = r[u];
            base += __popc(bal);
        }
    }
}

// Pivot rows restricted to the diagonal block: the panel's pivot rows are the first 64 rows not yet
// pivoted, in order (the rows c0 .. c0+63 when every earlier panel did the same); A11's own partial
// pivoting (gj_a11_lu_kernel) orders them.  One warp.
__global__ void gj_local_rows_kernel(int c0, int panel, int nact, GjWork w, const int* act, int* act_next) {
    const int lane = threadIdx.x;
    for (int i = lane; i < 64; i += 32) {
        const int r = act[i];
        w.piv[i] = r;
        w.perm[c0 + i] = r;
        w.pflag[r] = panel + 1;
    }
    for (int i = 64 + lane; i < nact; i += 32) act_next[i - 64] = act[i];
}

// LU of the panel's pivot block A11 = G[piv, panel] with partial pivoting (row i of the
// factored block is row perm[i] of A11): unit L below the diagonal, U on and above it, and the
// reciprocals of U's diagonal in rdiag.  One CTA; a zero or non-finite pivot sets SLAB_DEV_NOTSPD.
template <typename T>
__global__ void __launch_bounds__(256) gj_a11_lu_kernel(const T* __restrict__ G, int64_t ld, int c0, const int* piv,
                                                        T* LU, T* rdiag, int* perm, unsigned* status) {
    extern __shared__ unsigned char gj_smem[];
    T (*M)[65] = reinterpret_cast<T (*)[65]>(gj_smem);
    __shared__ int pr[64];
    __shared__ int pk;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        const int i = idx >> 6, j = idx & 63;
        M[i][j] = G[(int64_t)piv[i] * ld + c0 + j];
    }
    if (tid < 64) pr[tid] = tid;
    __syncthreads();
    for (int k = 0; k < 64; ++k) {
        if (tid < 32) {
            T best = T(-1);
            int bi = k;
            for (int i = k + tid; i < 64; i += 32) {
                const T v = fabs(M[i][k]);
                if (v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                if (!(best > T(0)) || !isfinite((double)best)) {
                    atomicOr(status, SLAB_DEV_NOTSPD);
                    M[bi][k] = T(1);
                }
                pk = bi;
                if (bi != k) { const int t2 = pr[k]; pr[k] = pr[bi]; pr[bi] = t2; }
            }
        }
        __syncthreads();
        const int p = pk;
        if (p != k && tid < 64) { const T t2 = M[k][tid]; M[k][tid] = M[p][tid]; M[p][tid] = t2; }
        __syncthreads();
        const T rp = T(1) / M[k][k];
        if (tid > k && tid < 64) M[tid][k] *= rp;                  // multipliers
        __syncthreads();
        const int r = 63 - k;
        for (int idx = tid; idx < r * r; idx += 256) {
            const int i = k + 1 + idx / r, j = k + 1 + idx % r;
            M[i][j] -= M[i][k] * M[k][j];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < 64 * 64; idx += 256) LU[idx] = M[idx >> 6][idx & 63];
    if (tid < 64) {
        rdiag[tid] = T(1) / M[tid][tid];
        perm[tid] = pr[tid];
    }
}

// blockIdx.y == 0: X = A11^{-1} G[piv, col0 .. col0+63] for 64 columns of the rest (cols >= c0+64),
// written to G[piv, cols] and to XT[col - (c0+64)][0..63].
// blockIdx.y == 1: Pbuf[r][0..63] = G[r][panel] for the top rows (0 for this panel's pivots)
// and the bottom rows.
template <typename T>
__global__ void __launch_bounds__(256) gj_panel_apply_kernel(T* Gt, int64_t ldt, const T* __restrict__ Gb,
                                                             int64_t ldb, int sp, int wt, int c0, int panel,
                                                             const int* piv, const int* pflag,
                                                             const T* __restrict__ LU, const T* __restrict__ rdiag,
                                                             const int* __restrict__ perm, T* XT, T* Pbuf) {
    extern __shared__ unsigned char gj_smem[];
    T (*Ai)[65] = reinterpret_cast<T (*)[65]>(gj_smem);
    T (*Bc)[65] = Ai + 64;
    const int tid = threadIdx.x;
    if (blockIdx.y == 1) {
        const int64_t rows = 2 * (int64_t)sp;
        for (int64_t idx = (int64_t)blockIdx.x * 256 + tid; idx < rows * 64; idx += (int64_t)gridDim.x * 256) {
            const int r = (int)(idx >> 6), c = (int)(idx & 63);
            T v;
            if (r < sp) v = pflag[r] == panel + 1 ? T(0) : Gt[(int64_t)r * ldt + c0 + c];
            else v = Gb[(int64_t)(r - sp) * ldb + c0 + c];
            Pbuf[idx] = v;
        }
        return;
    }
    const int cb = c0 + 64 + blockIdx.x * 64;           // first column of this block
    if (cb >= wt) return;
    const int nc = min(64, wt - cb);
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        const int i = idx >> 6, j = idx & 63;
        Ai[i][j] = LU[idx];
        Bc[i][j] = j < nc ? Gt[(int64_t)piv[perm[i]] * ldt + cb + j] : T(0);     // P B
    }
    __syncthreads();
    // X = U^{-1} L^{-1} P B, 64 columns at once
    for (int k = 0; k < 63; ++k) {                       // forward, unit L
        for (int idx = tid; idx < (63 - k) * 64; idx += 256) {
            const int i = k + 1 + (idx >> 6), j = idx & 63;
            Bc[i][j] -= Ai[i][k] * Bc[k][j];
        }
        __syncthreads();
    }
    for (int k = 63; k >= 0; --k) {                      // backward
        if (tid < 64) Bc[k][tid] *= rdiag[k];
        __syncthreads();
        for (int idx = tid; idx < k * 64; idx += 256) {
            const int i = idx >> 6, j = idx & 63;
            Bc[i][j] -= Ai[i][k] * Bc[k][j];
        }
        __syncthreads();
    }
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        const int i = idx >> 6, j = idx & 63;            // row of X, column in block
        if (j < nc) Gt[(int64_t)piv[i] * ldt + cb + j] = Bc[i][j];
    }
    for (int idx = tid; idx < 64 * 64; idx += 256) {
        const int j = idx >> 6, i = idx & 63;            // XT row = column, 64 consecutive i
        if (j < nc) XT[(int64_t)(cb - c0 - 64 + j) * 64 + i] = Bc[i][j];
    }
}

// Build the augmented system of interface j.  S comes from Tb[0] (j = 0) or from the bottom
// right block of the previous elimination (copied before the bottom block is rebuilt).
template <typename T>
__global__ void gj_fill_top_kernel(T* Gt, int sp, int wt, const T* __restrict__ S, int64_t lds,
                                   const T* __restrict__ T12) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)sp * wt) return;
    const int i = (int)(idx / wt), c = (int)(idx % wt);
    T v;
    if (c < sp) v = S[(int64_t)i * lds + c];
    else if (T12 && c < 2 * sp) v = T12[(int64_t)i * sp + (c - sp)];
    else v = (c - (wt - sp)) == i ? T(1) : T(0);
    Gt[idx] = v;
}

// Bottom rows [T_{j+1,j} | T_{j+1,j+1}]: T21 given (nonsymmetric kind), else T_{j,j+1}^T from T12.
template <typename T>
__global__ void gj_fill_bottom_kernel(T* Gb, int sp, const T* __restrict__ T12, const T* __restrict__ T22,
                                      const T* __restrict__ T21) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)sp * 2 * sp) return;
    const int i = (int)(idx / (2 * sp)), c = (int)(idx % (2 * sp));
    Gb[idx] = c < sp ? (T21 ? T21[(int64_t)i * sp + c] : T12[(int64_t)c * sp + i]) : T22[(int64_t)i * sp + (c - sp)];
}

// Sinv[i] = Gt[perm[i]][wt-sp ..], W[i] = Gt[perm[i]][sp .. 2sp) (W optional)
template <typename T>
__global__ void gj_gather_kernel(const T* __restrict__ Gt, int sp, int wt, const int* perm, T* Sinv, T* W) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)sp * sp) return;
    const int i = (int)(idx / sp), c = (int)(idx % sp);
    const T* row = Gt + (int64_t)perm[i] * wt;
    Sinv[idx] = row[wt - sp + c];
    if (W) W[idx] = row[sp + c];
}

template <typename T>
__global__ void gj_init_rows_kernel(int* act, int* pflag, int sp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < sp) { act[i] = i; pflag[i] = 0; }
}

// Batched C_b = beta C_b + alpha A_b B_b^T, b < batch, with element strides sA, sB, sC.
template <typename T>
slab_status gemm_tn_batched(slab_handle* h, int cls, int M, int N, int K, T alpha, const T* A, int64_t lda,
                            int64_t sA, const T* B, int64_t ldb, int64_t sB, T beta, T* C, int64_t ldc,
                            int64_t sC, int transC, int lower_only, int batch, int triA = 0);

template <>
slab_status gemm_tn_batched<float>(slab_handle* h, int cls, int M, int N, int K, float alpha, const float* A,
                                   int64_t lda, int64_t sA, const float* B, int64_t ldb, int64_t sB, float beta,
                                   float* C, int64_t ldc, int64_t sC, int transC, int lower_only, int batch, int triA) {
    // a factor product whose operand splits do not fit the FP16 work buffer runs on slices of the
    // batch that do, rather than falling back to the slower 3xTF32 product
    if (batch > 1 && h->w16 && !h->tf32_now && K % 64 == 0 &&
        (cls == KC_SYRK || cls == KC_TRAIL || cls == KC_ASSEMBLE)) {
        const bool shared = A == B && lda == ldb && sA == sB && N <= M;
        if (f16x3_work_bytes(M, N, K, batch, shared) > h->w16_bytes) {
            int bc = batch;
            while (bc > 1 && f16x3_work_bytes(M, N, K, bc, shared) > h->w16_bytes) bc = (bc + 1) / 2;
            if (f16x3_work_bytes(M, N, K, bc, shared) <= h->w16_bytes) {
                for (int b0 = 0; b0 < batch; b0 += bc) {
                    const int nb = std::min(bc, batch - b0);
                    const slab_status st = gemm_tn_batched<float>(h, cls, M, N, K, alpha, A + b0 * sA, lda, sA,
                                                                  B + b0 * sB, ldb, sB, beta, C + b0 * sC, ldc, sC,
                                                                  transC, lower_only, nb, triA);
                    if (st) return st;
                }
                return SLAB_OK;
            }
        }
    }
    SLAB_PROF(h, cls);
    if (skinny_ok(N, K, A, lda, sA, B, ldb, sB, lower_only))
        return launch_skinny(h, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, transC, batch);
    TcGemmArgs g;
    g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta;
    g.A = A; g.lda = lda; g.B = B; g.ldb = ldb; g.C = C; g.ldc = ldc;
    g.transC = transC; g.split = h->tf32_now ? 0 : 1; g.lower_only = lower_only;
    g.batch = batch; g.sA = sA; g.sB = sB; g.sC = sC;
    g.ksplit = 1; g.part = nullptr;
    g.w16 = nullptr; g.w16_bytes = 0;
    g.triA = triA;
    if (use_f16x3(h, cls, g)) {
        // FP16 three-product path (factor products)
    } else if (N <= 64 && !lower_only && h->wPart) {     // skinny batches that leave SMs idle: split K as well
        const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + 63) / 64) * batch;
        const int64_t cap = (int64_t)splitk_part_bytes(h->td.s_pad) / sizeof(float);
        int ks = 1;
        while (2 * ks <= SLAB_SPLITK && tiles * ks < 148 && K % (2 * ks * 32) == 0 &&
               (int64_t)2 * ks * batch * M * N <= cap)
            ks *= 2;
        g.ksplit = ks;
        g.part = (float*)h->wPart;
    }
    const slab_status st = tc_gemm(h->stream, g, h->dstatus);
    if (st == SLAB_ECUDA && h->err == SLAB_OK) h->err = SLAB_ECUDA;
    prof_extra(h, cls, tc_gemm_extra_launches(g));
    return st;
}

template <>
slab_status gemm_tn_batched<double>(slab_handle* h, int cls, int M, int N, int K, double alpha, const double* A,
                                    int64_t lda, int64_t sA, const double* B, int64_t ldb, int64_t sB,
                                    double beta, double* C, int64_t ldc, int64_t sC, int transC, int lower_only,
                                    int batch, int /*triA*/) {
    SLAB_PROF(h, cls);
    dim3 grid((N + TL - 1) / TL, (M + TL - 1) / TL, batch);
    gemm_tn_kernel<double><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, transC,
                                                        lower_only, sA, sB, sC);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

}  // namespace

// Indefinite kind: Algorithm 1 as printed, S_1 = T_11, S_{j+1} = T_{j+1,j+1} - T_{j+1,j} W_j with
// W_j = S_j^{-1} T_{j,j+1}, all three from one blocked Gauss-Jordan elimination of the augmented
// system (see above).  Stored: S_j^{-1} (in Linv), W_j (in Y) and T_{j+1,j} (in ToT).
// Work: Gt, Gb in Fct; Pbuf, XT, A11^{-1} and the pivot bookkeeping in gjw.
template <typename T>
slab_status sweep_factor_indef(slab_handle* h) {
    const int NI = h->td.NI, sp = h->td.s_pad, nt = h->nt;
    const int64_t blk = (int64_t)sp * sp;
    T* Tb = (T*)h->Tb;
    T* To = (T*)h->To;
    T* ToT = (T*)h->ToT;
    T* Tl = (T*)h->Tl;                   // nonsymmetric kind: T_{q+1,q} as assembled (else null)
    T* Sinv = (T*)h->Linv;
    T* Wn = (T*)h->Y;
    T* Gt = (T*)h->Fct;                  // sp x 3sp
    T* Gb = Gt + 3 * blk;                // sp x 2sp
    char* wb = (char*)h->gjw;
    T* Pbuf = (T*)wb;                    wb += (size_t)2 * sp * 64 * sizeof(T);
    T* XT = (T*)wb;                      wb += (size_t)3 * sp * 64 * sizeof(T);
    T* A11lu = (T*)wb;                   wb += (size_t)64 * 64 * sizeof(T);
    T* rdiag = (T*)wb;                   wb += (size_t)64 * sizeof(T);
    int* lperm = (int*)wb;               wb += (size_t)64 * sizeof(int);
    GjWork w;
    int* act0 = (int*)wb;                wb += (size_t)2 * sp * sizeof(int);
    w.act = act0;
    w.perm = (int*)wb;                   wb += (size_t)sp * sizeof(int);
    w.pflag = (int*)wb;                  wb += (size_t)sp * sizeof(int);
    const int nodes = gj_nodes((sp + GJ_LEAF - 1) / GJ_LEAF);
    w.cand = (int*)wb;                   wb += (size_t)nodes * 64 * sizeof(int);
    w.tick = (unsigned*)wb;              wb += (size_t)nodes * sizeof(unsigned);
    w.piv = (int*)wb;
    const size_t tsmem = (size_t)GJ_WARPS * GJ_LEAF * 65 * sizeof(float);
    const size_t ismem = (size_t)64 * 65 * sizeof(T);
    const size_t asmem = (size_t)2 * 64 * 65 * sizeof(T);
    SLAB_CK(h, cudaFuncSetAttribute(gj_tournament_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tsmem));
    SLAB_CK(h, cudaFuncSetAttribute(gj_a11_lu_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)ismem));
    SLAB_CK(h, cudaFuncSetAttribute(gj_panel_apply_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)asmem));
    SLAB_CK(h, cudaMemsetAsync(w.tick, 0, (size_t)nodes * sizeof(unsigned), h->stream));
    slab_status st;
    for (int j = 0; j < NI; ++j) {
        const bool hasNext = j < NI - 1;
        const int wt = (hasNext ? 3 : 2) * sp;
        {
            SLAB_PROF(h, KC_OTHER);
            const int64_t n1 = (int64_t)sp * wt;
            gj_fill_top_kernel<T><<<(unsigned)((n1 + 255) / 256), 256, 0, h->stream>>>(
                Gt, sp, wt, j == 0 ? Tb : Gb + sp, j == 0 ? sp : 2 * sp, hasNext ? To + j * blk : nullptr);
            SLAB_CK_LAUNCH(h);
            if (hasNext) {
                const int64_t n2 = 2 * blk;
                gj_fill_bottom_kernel<T><<<(unsigned)((n2 + 255) / 256), 256, 0, h->stream>>>(
                    Gb, sp, To + j * blk, Tb + (j + 1) * blk, Tl ? Tl + j * blk : nullptr);
                SLAB_CK_LAUNCH(h);
            }
            gj_init_rows_kernel<T><<<(sp + 255) / 256, 256, 0, h->stream>>>(act0, w.pflag, sp);
            SLAB_CK_LAUNCH(h);
        }
        for (int kb = 0; kb < nt; ++kb) {
            const int c0 = kb * 64;
            const int nact = sp - c0;
            const int* act = act0 + (kb & 1) * sp;
            int* act_next = act0 + ((kb + 1) & 1) * sp;
            const int L = (nact + GJ_LEAF - 1) / GJ_LEAF;
            {
                SLAB_PROF(h, KC_PANEL);
                if (h->pivot_local)
                    gj_local_rows_kernel<<<1, 32, 0, h->stream>>>(c0, kb, nact, w, act, act_next);
                else
                    gj_tournament_kernel<T><<<(L + GJ_WARPS - 1) / GJ_WARPS, 32 * GJ_WARPS, tsmem, h->stream>>>(
                        Gt, wt, c0, kb, nact, w, act, act_next);
                SLAB_CK_LAUNCH(h);
                gj_a11_lu_kernel<T><<<1, 256, ismem, h->stream>>>(Gt, wt, c0, w.piv, A11lu, rdiag, lperm, h->dstatus);
                SLAB_CK_LAUNCH(h);
                const int ncol = wt - c0 - 64;
                dim3 grid((unsigned)std::max((ncol + 63) / 64, 64), 2);
                gj_panel_apply_kernel<T><<<grid, 256, asmem, h->stream>>>(Gt, wt, Gb, 2 * sp, sp, wt, c0, kb, w.piv,
                                                                     w.pflag, A11lu, rdiag, lperm, XT, Pbuf);
                SLAB_CK_LAUNCH(h);
            }
            // G[other, rest] -= Pbuf X : top rows over all remaining columns, bottom rows up to 2 sp
            const int nt_top = wt - c0 - 64;
            if ((st = gemm_tn<T>(h, KC_TRAIL, sp, nt_top, 64, T(-1), Pbuf, 64, XT, 64, T(1), Gt + c0 + 64, wt, 0, 0)))
                return st;
            const int nb_bot = 2 * sp - c0 - 64;
            if (hasNext && (st = gemm_tn<T>(h, KC_TRAIL, sp, nb_bot, 64, T(-1), Pbuf + (int64_t)sp * 64, 64, XT, 64,
                                            T(1), Gb + c0 + 64, 2 * sp, 0, 0)))
                return st;
            if (slab_debug()) {
                if (slab_debug_status(h, "interface elimination (interface, panel)", j, kb)) return SLAB_ESINGULAR;
                // pivot bookkeeping: distinct pivot rows drawn from the active list, act_next = act - piv
                std::vector<int> hp(64), ha(nact), hn(nact > 64 ? nact - 64 : 1);
                cudaMemcpy(hp.data(), w.piv, 64 * sizeof(int), cudaMemcpyDeviceToHost);
                cudaMemcpy(ha.data(), act, nact * sizeof(int), cudaMemcpyDeviceToHost);
                if (nact > 64) cudaMemcpy(hn.data(), act_next, (nact - 64) * sizeof(int), cudaMemcpyDeviceToHost);
                std::vector<char> inA(sp, 0), inP(sp, 0);
                bool bad = false;
                for (int r : ha) inA[r] = 1;
                for (int r : hp) { if (r < 0 || r >= sp || !inA[r] || inP[r]) bad = true; else inP[r] = 1; }
                size_t q = 0;
                for (int r : ha) if (!inP[r]) { if (q >= hn.size() || hn[q] != r) bad = true; ++q; }
                if (bad) {
                    std::fprintf(stderr, "slab: pivot bookkeeping inconsistent at (%d, %d)\n", j, kb);
                    return SLAB_ESINGULAR;
                }
            }
        }
        {
            SLAB_PROF(h, KC_OTHER);
            gj_gather_kernel<T><<<(unsigned)((blk + 255) / 256), 256, 0, h->stream>>>(Gt, sp, wt, w.perm,
                                                                                    Sinv + j * blk,
                                                                                    hasNext ? Wn + j * blk : nullptr);
            SLAB_CK_LAUNCH(h);
        }
        if (!Tl && hasNext && (st = transpose<T>(h, To + j * blk, ToT + j * blk, sp))) return st;   // T_{j+1,j}
        if (Tl) {                        // factors of the transposed sweep (A^T solves)
            if ((st = transpose<T>(h, Sinv + j * blk, (T*)h->SinvT + j * blk, sp))) return st;
            if (hasNext && (st = transpose<T>(h, Wn + j * blk, (T*)h->WT + j * blk, sp))) return st;
            if (hasNext && (st = transpose<T>(h, Tl + j * blk, (T*)h->TlT + j * blk, sp))) return st;
        }
    }
    return SLAB_OK;
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (D)src[i];
}

slab_status widen_to_double(slab_handle* h, const float* src, double* dst, int64_t n) {
    if (n <= 0) return SLAB_OK;
    SLAB_PROF(h, KC_OTHER);
    convert_kernel<float, double><<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, h->stream>>>(
        src, dst, n);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status narrow_to_float(slab_handle* h, const double* src, float* dst, int64_t n) {
    if (n <= 0) return SLAB_OK;
    SLAB_PROF(h, KC_OTHER);
    convert_kernel<double, float><<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, h->stream>>>(
        src, dst, n);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

// Bytes of the indefinite-kind Stage-2 work area (gjw).
size_t gj_work_bytes(int sp, size_t rsz) {
    const int nodes = gj_nodes((sp + GJ_LEAF - 1) / GJ_LEAF);
    return (size_t)(2 + 3) * sp * 64 * rsz + 64 * 64 * rsz + (size_t)4 * sp * sizeof(int) +
           (size_t)nodes * 64 * sizeof(int) + (size_t)nodes * sizeof(unsigned) + 64 * sizeof(int) + 64 * rsz +
           64 * sizeof(int) + 256;
}

// Algorithm 2 for the indefinite kind on X ([NI][kcap][s_pad]):
//   forward  z_j = S_j^{-1} f_j,  f_{j+1} -= T_{j+1,j} z_j;   backward  u_j = z_j - W_j u_{j+1}.
template <typename T>
slab_status sweep_solve_indef(slab_handle* h, int K) {
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    const int64_t vb = (int64_t)sp * h->kcap;
    T* Sinv = (T*)h->Linv;
    T* Wn = (T*)h->Y;
    T* ToT = h->Tl ? (T*)h->Tl : (T*)h->ToT;     // T_{j+1,j}
    T* X = (T*)h->wX;
    T* Z = (T*)h->wZ;
    slab_status st;
    for (int j = 0; j < NI; ++j) {
        if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(1), Sinv + j * blk, sp, X + j * vb, sp, T(0), Z + j * vb,
                             sp, 1, 0)))
            return st;
        if (j < NI - 1 && (st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(-1), ToT + j * blk, sp, Z + j * vb, sp,
                                           T(1), X + (j + 1) * vb, sp, 1, 0)))
            return st;
    }
    for (int j = NI - 1; j >= 0; --j) {
        SLAB_CK(h, cudaMemcpyAsync(X + j * vb, Z + j * vb, (size_t)K * sp * sizeof(T), cudaMemcpyDeviceToDevice,
                                   h->stream));
        if (j < NI - 1 && (st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(-1), Wn + j * blk, sp, X + (j + 1) * vb, sp,
                                           T(1), X + j * vb, sp, 1, 0)))
            return st;
    }
    return SLAB_OK;
}

// Algorithm 2 for T^T (the adjoint of the nonsymmetric kind) with the factors of T = L U, L block
// lower bidiagonal (S_j, T_{j+1,j}), U unit block upper bidiagonal (W_j): T^T = U^T L^T, so
//   forward  y_j = f_j - W_{j-1}^T y_{j-1};   backward  x_j = S_j^{-T} (y_j - T_{j+1,j}^T x_{j+1}),
// on X ([NI][kcap][s_pad]), result in X.
template <typename T>
slab_status sweep_solve_indef_transposed(slab_handle* h, int K) {
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    const int64_t vb = (int64_t)sp * h->kcap;
    T* SinvT = (T*)h->SinvT;
    T* WT = (T*)h->WT;
    T* TlT = (T*)h->TlT;
    T* X = (T*)h->wX;
    T* Z = (T*)h->wZ;
    slab_status st;
    for (int j = 1; j < NI; ++j)
        if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(-1), WT + (j - 1) * blk, sp, X + (j - 1) * vb, sp, T(1),
                             X + j * vb, sp, 1, 0)))
            return st;
    for (int j = NI - 1; j >= 0; --j) {
        if (j < NI - 1 && (st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(-1), TlT + j * blk, sp, Z + (j + 1) * vb, sp,
                                           T(1), X + j * vb, sp, 1, 0)))
            return st;
        if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(1), SinvT + j * blk, sp, X + j * vb, sp, T(0), Z + j * vb,
                             sp, 1, 0)))
            return st;
    }
    for (int j = 0; j < NI; ++j)
        SLAB_CK(h, cudaMemcpyAsync(X + j * vb, Z + j * vb, (size_t)K * sp * sizeof(T), cudaMemcpyDeviceToDevice,
                                   h->stream));
    return SLAB_OK;
}

// Factor-phase layout: Fct[j] = [S_j ; Y_j^T ; L_j^{-T}] (3 s_pad x s_pad; for the last j the
// L^{-T} block sits right below S), plus the transposed copies Lin[j] = L_j^{-1} and Yn[j] = Y_j
// for the solve products.
template <typename T>
slab_status sweep_factor(slab_handle* h) {
    if (h->kind == SLAB_HELMHOLTZ || h->kind == SLAB_CONVECTION) return sweep_factor_indef<T>(h);
    if (h->stage2) return cr_factor<T>(h);
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    T* Tb = (T*)h->Tb;
    T* To = (T*)h->To;
    T* F = (T*)h->Fct;
    T* Lin = (T*)h->Linv;
    T* Yn = (T*)h->Y;
    slab_status st;
    for (int j = 0; j < NI; ++j) {
        T* W = F + j * 3 * blk;
        const int hasY = j < NI - 1;
        T* S = W;
        T* Yt = W + blk;
        T* LT = W + (hasY ? 2 : 1) * blk;
        SLAB_CK(h, cudaMemcpyAsync(S, Tb + j * blk, blk * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
        if (j > 0) {           // S_j = T_jj - Y_{j-1}^T Y_{j-1}  (lower tiles)
            const T* Yp = F + (j - 1) * 3 * blk + blk;
            if ((st = gemm_tn<T>(h, KC_SYRK, sp, sp, sp, T(-1), Yp, sp, Yp, sp, T(1), S, sp, 0, 1))) return st;
        }
        {
            SLAB_PROF(h, KC_OTHER);
            if ((st = set_identity<T>(h, LT, sp, blk, 1))) return st;
        }
        if (hasY && (st = transpose<T>(h, To + j * blk, Yt, sp))) return st;      // T_{j+1,j}
        const int lt0 = (hasY ? 2 : 1) * sp;         // first row of the identity block
        if ((st = dense_tall_cholesky<T>(h, W, sp, lt0, 1, 0))) return st;
        if ((st = transpose<T>(h, LT, Lin + j * blk, sp))) return st;
        if (hasY && (st = transpose<T>(h, Yt, Yn + j * blk, sp))) return st;
    }
    return SLAB_OK;
}

// Algorithm 2 on the interface workspace X ([NI][kcap][s_pad], right-hand sides 0..K-1), result in X.
template <typename T>
slab_status sweep_solve(slab_handle* h, int K) {
    if (h->kind == SLAB_CONVECTION && h->transposed) return sweep_solve_indef_transposed<T>(h, K);
    if (h->kind == SLAB_HELMHOLTZ || h->kind == SLAB_CONVECTION) return sweep_solve_indef<T>(h, K);
    if (h->stage2) return cr_solve<T>(h, K);
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    const int64_t vb = (int64_t)sp * h->kcap;
    T* F = (T*)h->Fct;
    T* Lin = (T*)h->Linv;
    T* Yn = (T*)h->Y;
    T* X = (T*)h->wX;
    T* Z = (T*)h->wZ;
    slab_status st;
    for (int j = 0; j < NI; ++j) {        // forward: z_j = L_j^{-1} (f_j - Y_{j-1}^T z_{j-1})
        if (j > 0) {
            const T* Yt = F + (j - 1) * 3 * blk + blk;
            if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(-1), Yt, sp, Z + (j - 1) * vb, sp, T(1), X + j * vb, sp, 1, 0)))
                return st;
        }
        if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(1), Lin + j * blk, sp, X + j * vb, sp, T(0), Z + j * vb, sp, 1, 0,
                             1)))                 // L^{-1} is lower triangular
            return st;
    }
    for (int j = NI - 1; j >= 0; --j) {   // backward: u_j = L_j^{-T} (z_j - Y_j u_{j+1})
        if (j < NI - 1) {
            if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(-1), Yn + j * blk, sp, X + (j + 1) * vb, sp, T(1), Z + j * vb, sp,
                                 1, 0)))
                return st;
        }
        const T* LT = F + j * 3 * blk + (j < NI - 1 ? 2 : 1) * blk;
        if ((st = gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(1), LT, sp, Z + j * vb, sp, T(0), X + j * vb, sp, 1, 0,
                             2)))                 // L^{-T} is upper triangular
            return st;
    }
    return SLAB_OK;
}

// ------------------------------------------------------------------ odd-even elimination order
// The odd-even order for eliminating the blocks of T (Sec. 4, remark on the elimination order;
// conclusion).  Each level eliminates the blocks at odd positions among the remaining ones; the
// remaining blocks of level l are the multiples of 2^l, so the eliminated ones o = 2^l (2i+1) and
// their neighbours a = o - 2^l, c = o + 2^l (absent past the last block) are uniformly strided,
// and every step of a level is one batched launch.  With D the current diagonal blocks and
// E_i the current block coupling i to its right remaining neighbour:
//   L_o L_o^T = D_o,  P_o = L_o^{-1} E_a^T,  Q_o = L_o^{-1} E_o,
//   D_a -= P_o^T P_o,  D_c -= Q_o^T Q_o,  E_a <- -P_o^T Q_o.
// Stored per eliminated block: L^{-1} (Linv), L^{-T}, P^T, P, Q^T, Q.  Solve: forward
// y_o = L_o^{-1} b_o, b_a -= P_o^T y_o, b_c -= Q_o^T y_o level by level; the last block
// x = L^{-T} L^{-1} b; backward x_o = L_o^{-T} (y_o - P_o x_a - Q_o x_c).
struct CrLevel {
    int o0, step, nb, nc;     // first eliminated block, its neighbour distance, #eliminated, #with a c
};

static std::vector<CrLevel> cr_levels(int NI, int* last) {
    std::vector<CrLevel> L;
    int step = 1;
    while (step < NI) {                          // remaining: 0, step, 2 step, ... < NI
        const int nrem = (NI - 1) / step + 1;
        if (nrem < 2) break;
        CrLevel lv;
        lv.o0 = step;
        lv.step = step;
        lv.nb = nrem / 2;                        // positions 1, 3, 5, ... < nrem
        lv.nc = (nrem - 1) / 2;                  // those with position + 1 < nrem
        L.push_back(lv);
        step *= 2;
    }
    *last = 0;
    return L;
}

int cr_max_batch(int NI) {
    int last = 0;
    std::vector<CrLevel> L = cr_levels(NI, &last);
    int b = 1;
    for (auto& lv : L) b = std::max(b, lv.nb);
    return b;
}

// Cholesky with L^{-1} and L^{-T} of nb blocks D[o0 + i st] as one batch of tall eliminations
// [D ; I] in the work buffer (2 s_pad x s_pad per block).
template <typename T>
static slab_status cr_potrf_batch(slab_handle* h, int o0, int st_blk, int nb) {
    const int sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    T* D = (T*)h->crD;
    T* W = (T*)h->crW;
    T* LT = (T*)h->crLT;
    T* Lin = (T*)h->Linv;
    const int64_t sb = (int64_t)st_blk * blk;
    for (int i = 0; i < nb; ++i)
        SLAB_CK(h, cudaMemcpyAsync(W + i * 2 * blk, D + o0 * blk + i * sb, blk * sizeof(T), cudaMemcpyDeviceToDevice,
                                   h->stream));
    slab_status st;
    {
        SLAB_PROF(h, KC_OTHER);
        if ((st = set_identity<T>(h, W + blk, sp, 2 * blk, nb))) return st;
    }
    if ((st = dense_tall_cholesky<T>(h, W, sp, sp, nb, 2 * blk))) return st;
    for (int i = 0; i < nb; ++i)
        SLAB_CK(h, cudaMemcpyAsync(LT + o0 * blk + i * sb, W + i * 2 * blk + blk, blk * sizeof(T),
                                   cudaMemcpyDeviceToDevice, h->stream));
    return transpose_batched<T>(h, LT + o0 * blk, sb, Lin + o0 * blk, sb, sp, nb);
}

template <typename T>
slab_status cr_factor(slab_handle* h) {
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    T* D = (T*)h->crD;
    T* E = (T*)h->crE;
    T* Et = (T*)h->crW;                  // free between the batched Cholesky steps
    T* Lin = (T*)h->Linv;
    T* Pt = (T*)h->crPt;
    T* P = (T*)h->crP;
    T* Qt = (T*)h->crQt;
    T* Q = (T*)h->crQ;
    SLAB_CK(h, cudaMemcpyAsync(D, h->Tb, NI * blk * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
    if (NI > 1)
        SLAB_CK(h, cudaMemcpyAsync(E, h->To, (NI - 1) * blk * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
    int last = 0;
    const std::vector<CrLevel> levels = cr_levels(NI, &last);
    slab_status st;
    for (const CrLevel& lv : levels) {
        const int o0 = lv.o0, a0 = lv.o0 - lv.step, c0 = lv.o0 + lv.step, nb = lv.nb, nc = lv.nc;
        const int64_t sb = 2 * (int64_t)lv.step * blk;           // stride between consecutive o (and a, c)
        if ((st = cr_potrf_batch<T>(h, o0, 2 * lv.step, nb))) return st;
        // P_o^T = E_a L_o^{-T};  Q_o^T = E_o^T L_o^{-T}
        if ((st = gemm_tn_batched<T>(h, KC_SYRK, sp, sp, sp, T(1), E + a0 * blk, sp, sb, Lin + o0 * blk, sp, sb, T(0),
                                     Pt + o0 * blk, sp, sb, 0, 0, nb)))
            return st;
        if (nc > 0) {
            if ((st = transpose_batched<T>(h, E + o0 * blk, sb, Et, blk, sp, nc))) return st;
            if ((st = gemm_tn_batched<T>(h, KC_SYRK, sp, sp, sp, T(1), Et, sp, blk, Lin + o0 * blk, sp, sb, T(0),
                                         Qt + o0 * blk, sp, sb, 0, 0, nc)))
                return st;
        }
        // D_a -= P_o^T P_o (lower tiles)
        if ((st = gemm_tn_batched<T>(h, KC_SYRK, sp, sp, sp, T(-1), Pt + o0 * blk, sp, sb, Pt + o0 * blk, sp, sb, T(1),
                                     D + a0 * blk, sp, sb, 0, 1, nb)))
            return st;
        if (nc > 0) {
            // D_c -= Q_o^T Q_o (lower tiles);  E_a = -P_o^T Q_o
            if ((st = gemm_tn_batched<T>(h, KC_SYRK, sp, sp, sp, T(-1), Qt + o0 * blk, sp, sb, Qt + o0 * blk, sp, sb,
                                         T(1), D + c0 * blk, sp, sb, 0, 1, nc)))
                return st;
            if ((st = gemm_tn_batched<T>(h, KC_SYRK, sp, sp, sp, T(-1), Pt + o0 * blk, sp, sb, Qt + o0 * blk, sp, sb,
                                         T(0), E + a0 * blk, sp, sb, 0, 0, nc)))
                return st;
            if ((st = transpose_batched<T>(h, Qt + o0 * blk, sb, Q + o0 * blk, sb, sp, nc))) return st;
        }
        if ((st = transpose_batched<T>(h, Pt + o0 * blk, sb, P + o0 * blk, sb, sp, nb))) return st;
    }
    return cr_potrf_batch<T>(h, last, 1, 1);
}

template <typename T>
slab_status cr_solve(slab_handle* h, int K) {
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    const int64_t vb = (int64_t)sp * h->kcap;
    T* Lin = (T*)h->Linv;
    T* LT = (T*)h->crLT;
    T* Pt = (T*)h->crPt;
    T* P = (T*)h->crP;
    T* Qt = (T*)h->crQt;
    T* Q = (T*)h->crQ;
    T* X = (T*)h->wX;
    T* Z = (T*)h->wZ;
    int last = 0;
    const std::vector<CrLevel> levels = cr_levels(NI, &last);
    slab_status st;
    // out_i (K x sp, RHS-major) = beta out_i + alpha M_i v_i for the nbat strided blocks i;
    // a single product takes the split-K path; L^{-1} (lower) and L^{-T} (upper) are triangular
#define TRI(Mx) ((Mx) == Lin ? 1 : ((Mx) == LT ? 2 : 0))
#define PROD(Mx, m0, V, v0, OUT, w0, alpha_, beta_, nbat, sm, sv)                                                   \
    if ((st = (nbat) == 1                                                                                          \
                  ? gemm_tn<T>(h, KC_SOLVE_PROD, sp, K, sp, T(alpha_), Mx + (m0) * blk, sp, V + (v0) * vb, sp,      \
                               T(beta_), OUT + (w0) * vb, sp, 1, 0, TRI(Mx))                                      \
                  : gemm_tn_batched<T>(h, KC_SOLVE_PROD, sp, K, sp, T(alpha_), Mx + (m0) * blk, sp, (sm) * blk,    \
                                       V + (v0) * vb, sp, (sv) * vb, T(beta_), OUT + (w0) * vb, sp, (sv) * vb, 1, \
                                       0, (nbat), TRI(Mx))))                                                       \
    return st
    for (const CrLevel& lv : levels) {
        const int o0 = lv.o0, a0 = lv.o0 - lv.step, c0 = lv.o0 + lv.step, s2 = 2 * lv.step;
        PROD(Lin, o0, X, o0, Z, o0, 1, 0, lv.nb, s2, s2);
        PROD(Pt, o0, Z, o0, X, a0, -1, 1, lv.nb, s2, s2);
        if (lv.nc > 0) PROD(Qt, o0, Z, o0, X, c0, -1, 1, lv.nc, s2, s2);
    }
    PROD(Lin, last, X, last, Z, last, 1, 0, 1, 1, 1);
    PROD(LT, last, Z, last, X, last, 1, 0, 1, 1, 1);
    for (size_t l = levels.size(); l-- > 0;) {
        const CrLevel& lv = levels[l];
        const int o0 = lv.o0, a0 = lv.o0 - lv.step, c0 = lv.o0 + lv.step, s2 = 2 * lv.step;
        PROD(P, o0, X, a0, Z, o0, -1, 1, lv.nb, s2, s2);
        if (lv.nc > 0) PROD(Q, o0, X, c0, Z, o0, -1, 1, lv.nc, s2, s2);
        PROD(LT, o0, Z, o0, X, o0, 1, 0, lv.nb, s2, s2);
    }
#undef PROD
#undef TRI
    return SLAB_OK;
}

template slab_status sweep_factor<float>(slab_handle*);
template slab_status sweep_factor<double>(slab_handle*);
template slab_status sweep_solve<float>(slab_handle*, int);
template slab_status sweep_solve<double>(slab_handle*, int);
template slab_status cr_factor<float>(slab_handle*);
template slab_status cr_factor<double>(slab_handle*);
template slab_status cr_solve<float>(slab_handle*, int);
template slab_status cr_solve<double>(slab_handle*, int);

// ---------------------------------------------------------------- exported dense helpers
namespace {
// out[c][r] = in[r][c] for a rows x cols block (leading dimensions ldin, ldout), batched by blockIdx.z
template <typename T>
__global__ void __launch_bounds__(256) transpose_rect_kernel(const T* __restrict__ in, int64_t ldin, int64_t sin,
                                                             T* __restrict__ out, int64_t ldout, int64_t sout,
                                                             int rows, int cols) {
    transpose_tile64<T>(in + (int64_t)blockIdx.z * sin, ldin, out + (int64_t)blockIdx.z * sout, ldout, rows, cols);
}

template <typename T>
__global__ void copy_batched_kernel(const T* __restrict__ in, int64_t sin, T* __restrict__ out, int64_t sout,
                                    int64_t n) {
    in += (int64_t)blockIdx.y * sin;
    out += (int64_t)blockIdx.y * sout;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) out[i] = in[i];
}

// The same copy in 16-byte units (both blocks 16-byte aligned, strides and length multiples of 16
// bytes), four loads in flight per thread before their stores.
__global__ void copy16_batched_kernel(const uint4* __restrict__ in, int64_t sin, uint4* __restrict__ out, int64_t sout,
                                      int64_t n) {
    in += (int64_t)blockIdx.y * sin;
    out += (int64_t)blockIdx.y * sout;
    const int64_t stride = (int64_t)gridDim.x * 256;
    int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = in[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; ++u) out[i + u * stride] = v[u];
    }
    for (; i < n; i += stride) out[i] = in[i];
}
}  // namespace

// Panel workspace (one 64 x 64 inverse per matrix of a batch); grown on demand during the factor.
// The factor allocates the panel inverses for its largest batch up front (factor_create); a
// larger request (direct use of the tall Cholesky) grows them.
static slab_status ensure_panel_work(slab_handle* h, size_t bytes) {
    if (h->pnl_bytes >= bytes) return SLAB_OK;
    if (h->pnl && !h->arena) cudaFree(h->pnl);         // waits for the work that may still read it
    h->pnl = nullptr;
    h->pnl_bytes = 0;
    const slab_status st = slab_dalloc(h, &h->pnl, bytes);
    if (st) return st;
    h->pnl_bytes = bytes;
    return SLAB_OK;
}

template <typename T>
slab_status dense_gemm(slab_handle* h, int cls, int M, int N, int K, T alpha, const T* A, int64_t lda, int64_t sA,
                       const T* B, int64_t ldb, int64_t sB, T beta, T* C, int64_t ldc, int64_t sC, int transC,
                       int lower_only, int batch, int triA) {
    if (batch <= 0 || M <= 0 || N <= 0) return SLAB_OK;
    if (batch == 1) return gemm_tn<T>(h, cls, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, transC, lower_only, triA);
    return gemm_tn_batched<T>(h, cls, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, transC, lower_only,
                              batch, triA);
}

template <typename T>
slab_status dense_transpose(slab_handle* h, const T* in, int64_t ldin, int64_t sin, T* out, int64_t ldout,
                            int64_t sout, int rows, int cols, int batch) {
    if (batch <= 0 || rows <= 0 || cols <= 0) return SLAB_OK;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        dim3 grid((cols + 63) / 64, (rows + 63) / 64, nb);
        SLAB_PROF(h, KC_OTHER);
        transpose_rect_kernel<T><<<grid, 256, 0, h->stream>>>(in + b0 * sin, ldin, sin, out + b0 * sout, ldout, sout,
                                                              rows, cols);
        SLAB_CK_LAUNCH(h);
    }
    return SLAB_OK;
}

template <typename T>
slab_status dense_copy(slab_handle* h, const T* in, int64_t sin, T* out, int64_t sout, int64_t n, int batch) {
    if (batch <= 0 || n <= 0) return SLAB_OK;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        SLAB_PROF(h, KC_OTHER);
        const T* ib = in + b0 * sin;
        T* ob = out + b0 * sout;
        const bool v16 = ((uintptr_t)ib % 16 == 0) && ((uintptr_t)ob % 16 == 0) && (sin * sizeof(T)) % 16 == 0 &&
                         (sout * sizeof(T)) % 16 == 0 && (n * sizeof(T)) % 16 == 0;
        if (v16) {
            const int64_t n16 = n * (int64_t)sizeof(T) / 16;
            copy16_batched_kernel<<<dim3((unsigned)std::min<int64_t>((n16 + 1023) / 1024, 64), nb), 256, 0,
                                    h->stream>>>((const uint4*)ib, sin * (int64_t)sizeof(T) / 16, (uint4*)ob,
                                                 sout * (int64_t)sizeof(T) / 16, n16);
        } else {
            copy_batched_kernel<T><<<dim3((unsigned)std::min<int64_t>((n + 255) / 256, 64), nb), 256, 0,
                                     h->stream>>>(ib, sin, ob, sout, n);
        }
        SLAB_CK_LAUNCH(h);
    }
    return SLAB_OK;
}

// Cholesky of the leading ncols x ncols block of a batch of tall matrices (row-major, ld = ncols,
// bstride apart) whose rows below are eliminated with it: rows [ncols, ident0) receive B^T L^{-T},
// rows [ident0, ident0 + ncols), which must hold the identity, receive L^{-T}.
// Identity row ident0 + r is zero in the columns left of r until column r is eliminated, so the
// columns [0, c) only ever touch rows [0, ident0 + c).
//
// Recursive column bisection (right-looking at every level): factor the left half of a column
// range, apply its one update to the right half -- C[c0:, c0:c1] -= P P[:c1-c0]^T with P the left
// half's columns and K = the left half's width -- then factor the right half.  64-column panels
// are the leaves (panel_diag_kernel factors the diagonal tile once, panel_apply_kernel scales the
// tiles below by its inverse).  Each level reads and writes the trailing matrix once, so the
// trailing updates stream it about log2(ncols / 64) times in all, and most of their flops fall in
// products with a large K.
namespace {

// C[c0 : rows, c0 : c1] -= W[c0 : rows, k0 : k1] W[c0 : c1, k0 : k1]^T (lower tiles of the square
// part), for every matrix of the batch.  Where the FP16 three-product work buffer of the factor is
// too small for the whole batch, the product runs on slices of the batch, or of K for one matrix.
template <typename T>
slab_status tall_update(slab_handle* h, T* W, int ncols, int rows, int c0, int c1, int k0, int k1, int batch,
                        int64_t bstride) {
    const int M = rows - c0, N = c1 - c0;
    int bchunk = batch, kchunk = k1 - k0;
    if (sizeof(T) == 4 && h->w16 && !h->tf32_now) {
        while (bchunk > 1 && f16x3_work_bytes(M, N, kchunk, bchunk, true) > h->w16_bytes) bchunk = (bchunk + 1) / 2;
        while (kchunk > TL && f16x3_work_bytes(M, N, kchunk, bchunk, true) > h->w16_bytes)
            kchunk = (kchunk / TL + 1) / 2 * TL;
    }
    slab_status st;
    for (int b0 = 0; b0 < batch; b0 += bchunk) {
        const int nb = std::min(bchunk, batch - b0);
        T* Wb = W + (int64_t)b0 * bstride;
        for (int ka = k0; ka < k1; ka += kchunk) {
            const int kw = std::min(kchunk, k1 - ka);
            const T* P = Wb + (int64_t)c0 * ncols + ka;
            if ((st = dense_gemm<T>(h, KC_TRAIL, M, N, kw, T(-1), P, ncols, bstride, P, ncols, bstride, T(1),
                                    Wb + (int64_t)c0 * ncols + c0, ncols, bstride, 0, 1, nb)))
                return st;
        }
    }
    return SLAB_OK;
}

// Whether a panel launch of `ctas` CTAs with one extra 64 x 64 tile of shared memory runs in one wave
// on the 152 SMs (two CTAs per SM in FP32, one in FP64): then every CTA can factor the diagonal
// tile itself and the separate diagonal launch is saved.
inline bool one_wave(int64_t ctas, size_t elem) { return ctas <= (elem == 4 ? 2 : 1) * 152; }

template <typename T>
slab_status tall_panel(slab_handle* h, T* W, int ncols, int ident0, int kb, int batch, int64_t bstride, size_t smem) {
    const int rows = ident0 + (kb + 1) * TL;
    const int nrt = rows / TL - kb - 1;
    T* Lw = (T*)h->pnl;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        if (nrt > 0 && one_wave((int64_t)nrt * nb, sizeof(T))) {
            SLAB_PROF(h, KC_PANEL);
            SLAB_CK(h, launch_pdl(panel_apply_kernel<T, true>, dim3(nrt, nb), dim3(256), smem + TL * PTP * sizeof(T),
                                  h->stream, W + b0 * bstride, (int64_t)ncols, kb, bstride, (const T*)Lw,
                                  h->dstatus));
            SLAB_CK_LAUNCH(h);
            continue;
        }
        {
            SLAB_PROF(h, KC_PANEL);
            SLAB_CK(h, launch_pdl(panel_diag_kernel<T>, dim3(1, nb), dim3(256), smem, h->stream, W + b0 * bstride,
                                  (int64_t)ncols, kb, h->dstatus, bstride, Lw));
            SLAB_CK_LAUNCH(h);
        }
        if (nrt > 0) {
            SLAB_PROF(h, KC_PANEL);
            SLAB_CK(h, launch_pdl(panel_apply_kernel<T, false>, dim3(nrt, nb), dim3(256), smem, h->stream,
                                  W + b0 * bstride, (int64_t)ncols, kb, bstride, (const T*)Lw, h->dstatus));
            SLAB_CK_LAUNCH(h);
        }
    }
    return SLAB_OK;
}

// Panels kb and kb+1 (kb+1 < ncols / 64), all updates from the columns left of kb applied: three
// launches -- panel_diag_kernel(kb), panel_pair_kernel(kb) (panel kb scaled, its update of panel
// kb+1, panel kb+1's diagonal factored), panel_apply_kernel(kb+1) -- instead of a panel, a product
// and a panel; one (panel_pair_full_kernel) where the row tiles fit in one wave.
template <typename T>
slab_status tall_pair(slab_handle* h, T* W, int ncols, int ident0, int kb, int batch, int64_t bstride, size_t smem) {
    const int nrt0 = (ident0 + (kb + 1) * TL) / TL - kb - 1;      // row tiles below the diagonal, panel kb
    const int nrt1 = (ident0 + (kb + 2) * TL) / TL - kb - 2;      // and panel kb+1
    const size_t psmem = 4 * TL * PTP * sizeof(T);
    T* Lw = (T*)h->pnl;
    for (int b0 = 0; b0 < batch; b0 += 65535) {
        const int nb = std::min(65535, batch - b0);
        T* Lw2 = Lw + (int64_t)nb * TL * TL;
        SLAB_PROF(h, KC_PANEL);
        if (ident0 % TL == 0 && nrt1 == nrt0 && one_wave((int64_t)(nrt0 + 1) * nb, sizeof(T))) {
            SLAB_CK(h, launch_pdl(panel_pair_full_kernel<T>, dim3(nrt0 + 1, nb), dim3(256), psmem + TL * PTP * sizeof(T),
                                  h->stream, W + b0 * bstride, (int64_t)ncols, kb, bstride, h->dstatus));
            SLAB_CK_LAUNCH(h);
            continue;
        }
        if (one_wave((int64_t)nrt0 * nb, sizeof(T))) {
            SLAB_CK(h, launch_pdl(panel_pair_kernel<T, true>, dim3(nrt0, nb), dim3(256), psmem + TL * PTP * sizeof(T),
                                  h->stream, W + b0 * bstride, (int64_t)ncols, kb, bstride, (const T*)Lw, Lw2,
                                  h->dstatus));
            SLAB_CK_LAUNCH(h);
        } else {
            SLAB_CK(h, launch_pdl(panel_diag_kernel<T>, dim3(1, nb), dim3(256), smem, h->stream, W + b0 * bstride,
                                  (int64_t)ncols, kb, h->dstatus, bstride, Lw));
            SLAB_CK_LAUNCH(h);
            SLAB_CK(h, launch_pdl(panel_pair_kernel<T, false>, dim3(nrt0, nb), dim3(256), psmem, h->stream,
                                  W + b0 * bstride, (int64_t)ncols, kb, bstride, (const T*)Lw, Lw2, h->dstatus));
            SLAB_CK_LAUNCH(h);
            prof_extra(h, KC_PANEL, 1);
        }
        if (nrt1 > 0) {
            SLAB_CK(h, launch_pdl(panel_apply_kernel<T, false>, dim3(nrt1, nb), dim3(256), smem, h->stream,
                                  W + b0 * bstride, (int64_t)ncols, kb + 1, bstride, (const T*)Lw2, h->dstatus));
            SLAB_CK_LAUNCH(h);
            prof_extra(h, KC_PANEL, 1);
        }
    }
    return SLAB_OK;
}

// Panels [kb0, kb1), all updates from the columns left of kb0 already applied.
template <typename T>
slab_status tall_chol_range(slab_handle* h, T* W, int ncols, int ident0, int kb0, int kb1, int batch,
                            int64_t bstride, size_t smem) {
    if (kb1 - kb0 == 1) return tall_panel<T>(h, W, ncols, ident0, kb0, batch, bstride, smem);
    // the fused pair saves launches on the latency-bound critical path of small batches; large batches
    // fill the GPU anyway, and there its redundant tile products cost more than the launches it saves
    const int64_t tiles = (int64_t)batch * ((ident0 + (kb0 + 1) * TL) / TL - kb0 - 1);
    if (kb1 - kb0 == 2 && tiles <= 8 * 152) return tall_pair<T>(h, W, ncols, ident0, kb0, batch, bstride, smem);
    const int kbm = kb0 + (kb1 - kb0) / 2;
    slab_status st;
    if ((st = tall_chol_range<T>(h, W, ncols, ident0, kb0, kbm, batch, bstride, smem))) return st;
    if ((st = tall_update<T>(h, W, ncols, ident0 + kbm * TL, kbm * TL, kb1 * TL, kb0 * TL, kbm * TL, batch, bstride)))
        return st;
    return tall_chol_range<T>(h, W, ncols, ident0, kbm, kb1, batch, bstride, smem);
}

}  // namespace

template <typename T>
slab_status dense_tall_cholesky(slab_handle* h, T* W, int ncols, int ident0, int batch, int64_t bstride) {
    const size_t smem = 2 * TL * PTP * sizeof(T);
    SLAB_CK(h, cudaFuncSetAttribute(panel_diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int tile = (int)(TL * PTP * sizeof(T));
    SLAB_CK(h, cudaFuncSetAttribute(panel_apply_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    SLAB_CK(h, cudaFuncSetAttribute(panel_apply_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem + tile));
    SLAB_CK(h, cudaFuncSetAttribute(panel_pair_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    4 * tile));
    SLAB_CK(h, cudaFuncSetAttribute(panel_pair_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    5 * tile));
    SLAB_CK(h, cudaFuncSetAttribute(panel_pair_full_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 5 * tile));
    const int bchunk = std::min(batch, 65535);
    slab_status st;
    if ((st = ensure_panel_work(h, 2 * (size_t)bchunk * TL * TL * sizeof(T)))) return st;   // L^-1 of two panels
    const int nt = ncols / TL;
    if (nt <= 0) return SLAB_OK;
    return tall_chol_range<T>(h, W, ncols, ident0, 0, nt, batch, bstride, smem);
}

template slab_status dense_gemm<float>(slab_handle*, int, int, int, int, float, const float*, int64_t, int64_t,
                                       const float*, int64_t, int64_t, float, float*, int64_t, int64_t, int, int, int, int);
template slab_status dense_gemm<double>(slab_handle*, int, int, int, int, double, const double*, int64_t, int64_t,
                                        const double*, int64_t, int64_t, double, double*, int64_t, int64_t, int, int,
                                        int, int);
template slab_status dense_transpose<float>(slab_handle*, const float*, int64_t, int64_t, float*, int64_t, int64_t,
                                            int, int, int);
template slab_status dense_transpose<double>(slab_handle*, const double*, int64_t, int64_t, double*, int64_t,
                                             int64_t, int, int, int);
template slab_status dense_copy<float>(slab_handle*, const float*, int64_t, float*, int64_t, int64_t, int);
template slab_status dense_copy<double>(slab_handle*, const double*, int64_t, double*, int64_t, int64_t, int);
template slab_status dense_tall_cholesky<float>(slab_handle*, float*, int, int, int, int64_t);
template slab_status dense_tall_cholesky<double>(slab_handle*, double*, int, int, int, int64_t);
