// Stage 2: factorisation of the block-tridiagonal reduced matrix T
// (Sec. 4, Algorithm 1) and the sweeping solve (Algorithm 2).
//
// T is symmetric positive definite for the SPD kinds, so Algorithm 1's
// S_1 = T_11, S_{j+1} = T_{j+1,j+1} - T_{j+1,j} S_j^{-1} T_{j,j+1} is carried
// out as a block Cholesky: S_j = L_j L_j^T, Y_j = L_j^{-1} T_{j,j+1},
// S_{j+1} = T_{j+1,j+1} - Y_j^T Y_j.  The stored factors are L_j^{-1} and Y_j, so
// Algorithm 2 becomes products only:
//   forward   z_j = L_j^{-1} (f_j - Y_{j-1}^T z_{j-1})
//   backward  u_j = L_j^{-T} (z_j - Y_j u_{j+1}).
// L_j^{-1} and Y_j come out of one right-looking elimination of [S_j | T_{j,j+1} | I]
// in 64 x 64 tiles: per tile column a panel kernel (Cholesky of the diagonal
// tile, its inverse, and the panel / right-hand-side row products) and a
// trailing-update kernel.
#include "slab_internal.cuh"

namespace {

constexpr int TL = SLAB_TILE;   // 64
constexpr int TLP = TL + 1;

// C(64x64) += alpha * op(A) op(B) over K (multiple of 16); 256 threads, 4x4 per thread.
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

// C = beta C + alpha op(A) op(B), M and K multiples of 64, N arbitrary (<= ldc).
// tri: 0 full; 1 A lower triangular (k < (row tile + 1) * 64); 2 op(A) upper (k >= row tile * 64);
// lower_only: skip output tiles above the diagonal.
template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, T alpha, const T* A,
                                                   int64_t lda, const T* B, int64_t ldb, T beta,
                                                   T* C, int64_t ldc, int tri, int lower_only) {
    __shared__ T sA[16 * TLP];
    __shared__ T sB[16 * TLP];
    const int bj = blockIdx.x, bi = blockIdx.y;
    if (lower_only && bj > bi) return;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    int k0 = 0, k1 = K;
    if (tri == 1) k1 = min(K, (bi + 1) * TL);
    if (tri == 2) k0 = bi * TL;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    const T* Ab = TA ? A + (int64_t)bi * TL : A + (int64_t)bi * TL * lda;
    const T* Bb = TB ? B + (int64_t)bj * TL * ldb : B + (int64_t)bj * TL;
    const int ncols = min(TL, N - bj * TL);
    tile_gemm<T, TA, TB>(acc, Ab, lda, Bb, ldb, k0, k1, ncols, sA, sB);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = bi * TL + ty + 16 * a, c = bj * TL + tx + 16 * b;
            if (r < M && c < N) {
                T* p = C + (int64_t)r * ldc + c;
                *p = (beta == T(0) ? T(0) : beta * *p) + alpha * acc[a][b];
            }
        }
}

// Skinny product for the sweeping solve: C (M x N, N <= 64) = beta C + alpha op(A) B, A square
// M x K.  The K range is split over gridDim.y CTAs per 64-row tile; every CTA writes its partial
// tile to ws, and the last CTA of a tile (ticket counter) sums the partials in split order, so the
// result does not depend on scheduling.  tri as in gemm_kernel.
template <typename T, bool TA>
__global__ void __launch_bounds__(256) gemm_skinny_kernel(int M, int N, int K, T alpha, const T* A,
                                                          int64_t lda, const T* B, int64_t ldb, T beta,
                                                          T* C, int64_t ldc, int tri, T* ws,
                                                          unsigned* tickets) {
    __shared__ T sA[16 * TLP];
    __shared__ T sB[16 * TLP];
    __shared__ bool last;
    const int bi = blockIdx.x, sp = blockIdx.y, KS = gridDim.y;
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int kchunk = K / KS;
    int k0 = sp * kchunk, k1 = k0 + kchunk;
    if (tri == 1) k1 = min(k1, (bi + 1) * TL);
    if (tri == 2) k0 = max(k0, bi * TL);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    if (k0 < k1) {
        const T* Ab = TA ? A + (int64_t)bi * TL : A + (int64_t)bi * TL * lda;
        tile_gemm<T, TA, false>(acc, Ab, lda, B, ldb, k0, k1, N, sA, sB);
    }
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
            T* p = C + (int64_t)gr * ldc + c;
            *p = (beta == T(0) ? T(0) : beta * *p) + alpha * v;
        }
    }
    if (tid == 0) tickets[bi] = 0;
}

// Cholesky of the 64 x 64 tile in smem (lower, stride TLP), L in place, and Li = L^{-1}.
// 256 threads.  Blocked by 16 columns: warp 0 factors the 16 x 16 diagonal block with warp
// barriers only, one thread per row solves the panel below it, all threads update the rest.
// The inverse is formed blockwise: 16 x 16 diagonal inverses (one warp each, one lane per
// column), then block diagonals d = 1..3 from Li_IJ = -Li_II sum_{K=J}^{I-1} L_IK Li_KJ.
template <typename T>
__device__ void chol_inv_tile(T* S, T* Li, T* W, unsigned* status) {
    constexpr int NB = 16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int c0 = 0; c0 < TL; c0 += NB) {
        if (warp == 0) {
            for (int k = 0; k < NB; ++k) {
                const int kk = c0 + k;
                T d = S[kk * TLP + kk];
                const bool bad = !(d > T(0)) || !isfinite((double)d);
                if (bad) d = T(1);
                d = sqrt(d);
                __syncwarp();
                if (lane == k) {
                    S[kk * TLP + kk] = d;
                    if (bad) atomicOr(status, SLAB_DEV_NOTSPD);
                }
                if (lane > k && lane < NB) S[(c0 + lane) * TLP + kk] /= d;
                __syncwarp();
                if (lane > k && lane < NB) {
                    const T lik = S[(c0 + lane) * TLP + kk];
                    for (int j = k + 1; j <= lane; ++j) S[(c0 + lane) * TLP + c0 + j] -= lik * S[(c0 + j) * TLP + kk];
                }
                __syncwarp();
            }
        }
        __syncthreads();
        const int nrow = TL - c0 - NB;
        if (tid < nrow) {                       // row i: x L_bb^T = S[i, c0:c0+NB]
            const int i = c0 + NB + tid;
            T x[NB];
#pragma unroll
            for (int j = 0; j < NB; ++j) {
                T v = S[i * TLP + c0 + j];
#pragma unroll
                for (int l = 0; l < j; ++l) v -= x[l] * S[(c0 + j) * TLP + c0 + l];
                x[j] = v / S[(c0 + j) * TLP + c0 + j];
            }
#pragma unroll
            for (int j = 0; j < NB; ++j) S[i * TLP + c0 + j] = x[j];
        }
        __syncthreads();
        for (int idx = tid; idx < nrow * nrow; idx += blockDim.x) {
            const int i = c0 + NB + idx / nrow, j = c0 + NB + idx % nrow;
            if (j <= i) {
                T acc = T(0);
#pragma unroll
                for (int l = 0; l < NB; ++l) acc += S[i * TLP + c0 + l] * S[j * TLP + c0 + l];
                S[i * TLP + j] -= acc;
            }
        }
        __syncthreads();
    }
    // zero the strict upper triangle of Li, diagonal-block inverses (warp w < 4 owns block w)
    for (int idx = tid; idx < TL * TL; idx += blockDim.x) {
        const int i = idx / TL, j = idx % TL;
        if (j > i) Li[i * TLP + j] = T(0);
    }
    if (warp < 4 && lane < NB) {
        const int b0 = warp * NB, j = lane;
        for (int i = j; i < NB; ++i) {
            T v = (i == j) ? T(1) : T(0);
            for (int l = j; l < i; ++l) v -= S[(b0 + i) * TLP + b0 + l] * Li[(b0 + l) * TLP + b0 + j];
            Li[(b0 + i) * TLP + b0 + j] = v / S[(b0 + i) * TLP + b0 + i];
        }
        for (int i = 0; i < j; ++i) Li[(b0 + i) * TLP + b0 + j] = T(0);
    }
    __syncthreads();
    for (int dd = 1; dd < TL / NB; ++dd) {
        const int nblk = TL / NB - dd;         // blocks (I, J = I - dd)
        // W_IJ = sum_{K=J}^{I-1} L_IK Li_KJ
        for (int idx = tid; idx < nblk * NB * NB; idx += blockDim.x) {
            const int bI = dd + idx / (NB * NB), r = (idx / NB) % NB, c = idx % NB;
            const int bJ = bI - dd;
            T acc = T(0);
            for (int K = bJ; K < bI; ++K)
#pragma unroll
                for (int l = 0; l < NB; ++l)
                    acc += S[(bI * NB + r) * TLP + K * NB + l] * Li[(K * NB + l) * TLP + bJ * NB + c];
            W[(idx / (NB * NB)) * NB * NB + r * NB + c] = acc;
        }
        __syncthreads();
        for (int idx = tid; idx < nblk * NB * NB; idx += blockDim.x) {
            const int bI = dd + idx / (NB * NB), r = (idx / NB) % NB, c = idx % NB;
            const int bJ = bI - dd;
            T acc = T(0);
#pragma unroll
            for (int l = 0; l < NB; ++l)
                acc -= Li[(bI * NB + r) * TLP + bI * NB + l] * W[(idx / (NB * NB)) * NB * NB + l * NB + c];
            Li[(bI * NB + r) * TLP + bJ * NB + c] = acc;
        }
        __syncthreads();
    }
}

template <typename T>
struct SweepArgs {
    int nt, s_pad;
    T* Sw;        // S_j under elimination
    T* Yj;        // right-hand side block -> Y_j (may be null for the last block)
    T* Bj;        // identity -> L_j^{-1}
    unsigned* status;
    __device__ T* sw(int i, int c) const { return Sw + ((int64_t)i * TL) * s_pad + (int64_t)c * TL; }
    __device__ T* y(int i, int c) const { return Yj + ((int64_t)i * TL) * s_pad + (int64_t)c * TL; }
    __device__ T* bb(int i, int c) const { return Bj + ((int64_t)i * TL) * s_pad + (int64_t)c * TL; }
};

// Panel of tile column kb.  blockIdx.x: [0, nP) rows below the diagonal; [nP, nP+nY) Y row-block
// tiles; [nP+nY, ...) L^{-1} row-block tiles (columns <= kb).
template <typename T>
__global__ void __launch_bounds__(256) panel_kernel(SweepArgs<T> P, int kb, int hasY) {
    extern __shared__ unsigned char smem_raw[];
    T* S = reinterpret_cast<T*>(smem_raw);
    T* Li = S + TL * TLP;
    T* X = Li + TL * TLP;
    T* W = X + TL * TLP;                  // 3 x 16 x 16 scratch of the blocked inverse
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    const int nt = P.nt;
    const int nP = nt - kb - 1;
    const int nY = hasY ? nt : 0;
    int e = blockIdx.x;
    int kind, idx;
    if (e < nP) { kind = 0; idx = kb + 1 + e; }
    else if (e < nP + nY) { kind = 1; idx = e - nP; }
    else { kind = 2; idx = e - nP - nY; }
    const T* D = P.sw(kb, kb);
    for (int i = tid; i < TL * TL; i += 256) S[(i / TL) * TLP + i % TL] = D[(int64_t)(i / TL) * P.s_pad + i % TL];
    T* src = kind == 0 ? P.sw(idx, kb) : (kind == 1 ? P.y(kb, idx) : P.bb(kb, idx));
    for (int i = tid; i < TL * TL; i += 256) X[(i / TL) * TLP + i % TL] = src[(int64_t)(i / TL) * P.s_pad + i % TL];
    __syncthreads();
    chol_inv_tile<T>(S, Li, W, P.status);
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    if (kind == 0) {      // out = X Li^T
        for (int l = 0; l < TL; ++l) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = X[(ty + 16 * a) * TLP + l];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Li[(tx + 16 * b) * TLP + l];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
    } else {              // out = Li X
        for (int l = 0; l < TL; ++l) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = Li[(ty + 16 * a) * TLP + l];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = X[l * TLP + tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
            src[(int64_t)(ty + 16 * a) * P.s_pad + tx + 16 * b] = acc[a][b];
}

// Trailing update of tile column kb.  blockIdx.x enumerates: lower trailing tiles of S,
// then Y tiles (rows > kb, all columns), then L^{-1} tiles (rows > kb, columns <= kb).
template <typename T>
__global__ void __launch_bounds__(256) trailing_kernel(SweepArgs<T> P, int kb, int hasY) {
    __shared__ T sA[16 * TLP];
    __shared__ T sB[16 * TLP];
    const int nt = P.nt;
    const int R = nt - kb - 1;
    const int nS = R * (R + 1) / 2;
    const int nY = hasY ? R * nt : 0;
    int e = blockIdx.x;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    T* C;
    if (e < nS) {
        int ii = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
        while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
        while (ii * (ii + 1) / 2 > e) --ii;
        const int jj = e - ii * (ii + 1) / 2;
        const int i = kb + 1 + ii, i2 = kb + 1 + jj;
        tile_gemm<T, false, true>(acc, P.sw(i, kb), P.s_pad, P.sw(i2, kb), P.s_pad, 0, TL, TL, sA, sB);
        C = P.sw(i, i2);
    } else if (e < nS + nY) {
        e -= nS;
        const int i = kb + 1 + e / nt, c = e % nt;
        tile_gemm<T, false, false>(acc, P.sw(i, kb), P.s_pad, P.y(kb, c), P.s_pad, 0, TL, TL, sA, sB);
        C = P.y(i, c);
    } else {
        e -= nS + nY;
        const int i = kb + 1 + e / (kb + 1), c = e % (kb + 1);
        tile_gemm<T, false, false>(acc, P.sw(i, kb), P.s_pad, P.bb(kb, c), P.s_pad, 0, TL, TL, sA, sB);
        C = P.bb(i, c);
    }
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) C[(int64_t)(ty + 16 * a) * P.s_pad + tx + 16 * b] -= acc[a][b];
}

template <typename T>
__global__ void set_identity_kernel(T* B, int s_pad) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)s_pad * s_pad) return;
    B[idx] = (idx / s_pad == idx % s_pad) ? T(1) : T(0);
}

template <typename T, bool TA, bool TB>
slab_status gemm(slab_handle* h, int M, int N, int K, T alpha, const T* A, int64_t lda, const T* B,
                 int64_t ldb, T beta, T* C, int64_t ldc, int tri, int lower_only) {
    dim3 grid((N + TL - 1) / TL, M / TL);
    gemm_kernel<T, TA, TB><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,
                                                        tri, lower_only);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T, bool TA>
slab_status gemm_skinny(slab_handle* h, int M, int N, int K, T alpha, const T* A, int64_t lda, const T* B,
                        int64_t ldb, T beta, T* C, int64_t ldc, int tri) {
    int KS = K / 256;
    if (KS < 1) KS = 1;
    if (KS > SLAB_SPLITK) KS = SLAB_SPLITK;
    while (K % (KS * 16)) --KS;
    dim3 grid(M / TL, KS);
    gemm_skinny_kernel<T, TA><<<grid, 256, 0, h->stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tri,
                                                           (T*)h->wPart, h->wTickets);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

}  // namespace

template <typename T>
slab_status sweep_factor(slab_handle* h) {
    const int NI = h->td.NI, sp = h->td.s_pad, nt = h->nt;
    const int64_t blk = (int64_t)sp * sp;
    T* Tb = (T*)h->Tb;
    T* To = (T*)h->To;
    T* Linv = (T*)h->Linv;
    T* Y = (T*)h->Y;
    T* Sw = (T*)h->Swork;
    const size_t smem = (3 * TL * TLP + 3 * 16 * 16) * sizeof(T);
    SLAB_CK(h, cudaFuncSetAttribute(panel_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int j = 0; j < NI; ++j) {
        SLAB_CK(h, cudaMemcpyAsync(Sw, Tb + j * blk, blk * sizeof(T), cudaMemcpyDeviceToDevice, h->stream));
        if (j > 0) {
            slab_status st = gemm<T, true, false>(h, sp, sp, sp, T(-1), Y + (j - 1) * blk, sp,
                                                  Y + (j - 1) * blk, sp, T(1), Sw, sp, 0, 1);
            if (st) return st;
        }
        const int hasY = j < NI - 1;
        if (hasY)
            SLAB_CK(h, cudaMemcpyAsync(Y + j * blk, To + j * blk, blk * sizeof(T), cudaMemcpyDeviceToDevice,
                                       h->stream));
        set_identity_kernel<T><<<(unsigned)((blk + 255) / 256), 256, 0, h->stream>>>(Linv + j * blk, sp);
        SLAB_CK_LAUNCH(h);
        SweepArgs<T> P;
        P.nt = nt; P.s_pad = sp; P.Sw = Sw; P.Yj = hasY ? Y + j * blk : nullptr; P.Bj = Linv + j * blk;
        P.status = h->dstatus;
        for (int kb = 0; kb < nt; ++kb) {
            const int nP = nt - kb - 1, nY = hasY ? nt : 0, nB = kb + 1;
            panel_kernel<T><<<nP + nY + nB, 256, smem, h->stream>>>(P, kb, hasY);
            SLAB_CK_LAUNCH(h);
            const int R = nt - kb - 1;
            const int ntr = R * (R + 1) / 2 + (hasY ? R * nt : 0) + R * (kb + 1);
            if (ntr > 0) {
                trailing_kernel<T><<<ntr, 256, 0, h->stream>>>(P, kb, hasY);
                SLAB_CK_LAUNCH(h);
            }
        }
    }
    return SLAB_OK;
}

// Algorithm 2 on the interface workspace X ([NI][s_pad][kcap], columns 0..K-1), result in X.
template <typename T>
slab_status sweep_solve(slab_handle* h, int K) {
    const int NI = h->td.NI, sp = h->td.s_pad;
    const int64_t blk = (int64_t)sp * sp;
    const int64_t vb = (int64_t)sp * h->kcap;
    const int ld = h->kcap;
    T* Linv = (T*)h->Linv;
    T* Y = (T*)h->Y;
    T* X = (T*)h->wX;
    T* Z = (T*)h->wZ;
    slab_status st;
    for (int j = 0; j < NI; ++j) {        // forward: z_j = L_j^{-1} (f_j - Y_{j-1}^T z_{j-1})
        if (j > 0) {
            st = gemm_skinny<T, true>(h, sp, K, sp, T(-1), Y + (j - 1) * blk, sp, Z + (j - 1) * vb, ld, T(1),
                                      X + j * vb, ld, 0);
            if (st) return st;
        }
        st = gemm_skinny<T, false>(h, sp, K, sp, T(1), Linv + j * blk, sp, X + j * vb, ld, T(0), Z + j * vb,
                                   ld, 1);
        if (st) return st;
    }
    for (int j = NI - 1; j >= 0; --j) {   // backward: u_j = L_j^{-T} (z_j - Y_j u_{j+1})
        if (j < NI - 1) {
            st = gemm_skinny<T, false>(h, sp, K, sp, T(-1), Y + j * blk, sp, X + (j + 1) * vb, ld, T(1),
                                       Z + j * vb, ld, 0);
            if (st) return st;
        }
        st = gemm_skinny<T, true>(h, sp, K, sp, T(1), Linv + j * blk, sp, Z + j * vb, ld, T(0), X + j * vb, ld,
                                  2);
        if (st) return st;
    }
    return SLAB_OK;
}

template slab_status sweep_factor<float>(slab_handle*);
template slab_status sweep_factor<double>(slab_handle*);
template slab_status sweep_solve<float>(slab_handle*, int);
template slab_status sweep_solve<double>(slab_handle*, int);
