// Stage 1: elimination of the slab interiors (Sec. 3.1, Algorithm 3 first loop)
// and the parallel phases of Algorithm 4 (reduced load, eqs. f1-f5; interior
// back-solve, eq. usol_even).
//
// Each slab's interior block A_JJ is eliminated by cyclic reduction along y:
// the rows form a binary "ruler" tree (row c has height ctz(c)), and a launch
// eliminates every node of one height in every slab at once.  Node c merges
// the condensed systems of its two child segments through its separator row:
//   S   = D_c + R_alpha[bot,bot] + R_beta[top,top]            (m x m, SPD)
//   B   = couplings of row c to {top row, bot row, interface nodes of the segment}
//   L L^T = S,   Z = L^{-1} B,   R_merged = R_others - Z^T Z.
// Only the rows of R that belong to the top/bot rows are kept (the interface x
// interface part is summed later by the fused T assembly), so the per-node work
// is O(m^2 w) and the storage O(m s log s) per slab.
#include "slab_internal.cuh"

namespace {

constexpr int MAXM = SLAB_MAXM;
constexpr int SP = MAXM + 1;          // padded smem row stride for m x m
constexpr int SP2 = 2 * MAXM + 1;     // padded smem row stride for m x 2m
constexpr int TB_THREADS = 128;

template <typename T>
struct TreeArgs {
    int s, s_pad, m, H, NS, b, n;
    const double* AX;
    const double* AY;
    const double* DG;
    T* Linv;
    T* Ztb;
    T* Rtb;
    T* ZI;
    T* RI;
    T* Wtb;           // indefinite kind: W = S^{-1} B for the top/bot columns (else null)
    T* WI;            // indefinite kind: W = S^{-1} B for the interface columns, per height
    // Nonsymmetric kind only (else null).  A^T's couplings: AXT[y][x] = -h^2 A[(x+1,y),(x,y)],
    // AYT[y][x] = -h^2 A[(x,y+1),(x,y)] (AX / AY hold the forward ones, -h^2 A[(x,y),(x+1,y)] ...).
    // The factor stores, besides S^{-1} (Linv), C^T (Ztb, ZI: the couplings of the other nodes
    // into the separator) and W = S^{-1} B (Wtb, WI), the arrays of A^T's elimination: S^{-T}
    // (LinvT), B (ZtbT, ZIT) and V = S^{-T} C^T (WtbT, WIT); RIc holds the condensed
    // interface-row x top/bot-column couplings (the other orientation of RI).
    const double* AXT;
    const double* AYT;
    T* LinvT;
    T* ZtbT;
    T* WtbT;
    T* ZIT;
    T* WIT;
    T* RIc;
    unsigned* status;
    __device__ int64_t node(int t, int c) const { return (int64_t)t * (s + 1) + c; }
    __device__ T* linv(int t, int c) const { return Linv + node(t, c) * m * m; }
    __device__ T* ztb(int t, int c) const { return Ztb + node(t, c) * 2 * m * m; }
    __device__ T* rtb(int t, int c) const { return Rtb + node(t, c) * 4 * m * m; }
    __device__ T* zi(int t, int k, int side) const {
        return ZI + (((int64_t)t * H + k) * 2 + side) * m * s_pad;
    }
    __device__ T* wtb(int t, int c) const { return Wtb + node(t, c) * 2 * m * m; }
    __device__ T* wi(int t, int k, int side) const {
        return WI + (((int64_t)t * H + k) * 2 + side) * m * s_pad;
    }
    __device__ T* ri(int t, int k, int tb, int side) const {
        return RI + ((((int64_t)t * H + k) * 2 + tb) * 2 + side) * m * s_pad;
    }
    __device__ T* ric(int t, int k, int tb, int side) const {
        return RIc + ((((int64_t)t * H + k) * 2 + tb) * 2 + side) * m * s_pad;
    }
    __device__ T* per_height(T* base, int t, int k, int side) const {
        return base + (((int64_t)t * H + k) * 2 + side) * m * s_pad;
    }
    __device__ T* per_node(T* base, int t, int c, int blk) const { return base + node(t, c) * blk; }
};

template <typename T>
__device__ inline T dsqrt(T v) { return sqrt(v); }

// In-place Cholesky of the m x m matrix S (lower) and Li = L^{-1}; all threads of the block.
template <typename T>
__device__ void chol_inv_small(T* S, T* Li, int m, unsigned* status) {
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int k = 0; k < m; ++k) {
        if (tid == 0) {
            T d = S[k * SP + k];
            if (!(d > T(0)) || !isfinite((double)d)) {
                atomicOr(status, SLAB_DEV_NOTSPD);
                d = T(1);
            }
            S[k * SP + k] = dsqrt(d);
        }
        __syncthreads();
        if (tid > k && tid < m) S[tid * SP + k] /= S[k * SP + k];
        __syncthreads();
        const int r = m - k - 1;
        for (int idx = tid; idx < r * r; idx += nth) {
            const int i = k + 1 + idx / r, j = k + 1 + idx % r;
            if (j <= i) S[i * SP + j] -= S[i * SP + k] * S[j * SP + k];
        }
        __syncthreads();
    }
    for (int i = 0; i < m; ++i) {
        if (tid < m) {
            const int j = tid;
            T v = T(0);
            if (j <= i) {
                T acc = (i == j) ? T(1) : T(0);
                for (int l = j; l < i; ++l) acc -= S[i * SP + l] * Li[l * SP + j];
                v = acc / S[i * SP + i];
            }
            Li[i * SP + j] = v;
        }
        __syncthreads();
    }
}

// Inverse of the m x m matrix S (smem, stride SP; destroyed) into Si by Gauss-Jordan elimination
// of [S | I] with partial pivoting (first row of largest |s_ik| wins); all threads of the block.
// A zero or non-finite pivot sets SLAB_DEV_NOTSPD and continues with 1.
template <typename T>
__device__ void gj_inv_small(T* S, T* Si, int m, unsigned* status) {
    __shared__ int piv;
    __shared__ T prow;
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int idx = tid; idx < m * m; idx += nth) Si[(idx / m) * SP + idx % m] = (idx / m == idx % m) ? T(1) : T(0);
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (tid < 32) {                                  // pivot search in column k, rows k..m-1
            T best = T(-1);
            int bi = k;
            for (int i = k + tid; i < m; i += 32) {
                const T v = fabs(S[i * SP + k]);
                if (v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                piv = bi;
                const T pv = S[bi * SP + k];
                if (!(best > T(0)) || !isfinite((double)pv)) {
                    atomicOr(status, SLAB_DEV_NOTSPD);
                    prow = T(1);
                } else {
                    prow = T(1) / pv;
                }
            }
        }
        __syncthreads();
        const int p = piv;
        const T rp = prow;
        if (p != k)
            for (int j = tid; j < 2 * m; j += nth) {     // swap rows k and p of [S | Si]
                T* a = j < m ? S + k * SP + j : Si + k * SP + (j - m);
                T* b = j < m ? S + p * SP + j : Si + p * SP + (j - m);
                const T tmp = *a; *a = *b; *b = tmp;
            }
        __syncthreads();
        for (int j = tid; j < 2 * m; j += nth) {         // scale the pivot row
            if (j < m) S[k * SP + j] *= rp;
            else Si[k * SP + (j - m)] *= rp;
        }
        __syncthreads();
        for (int idx = tid; idx < m * 2 * m; idx += nth) {
            const int i = idx / (2 * m), j = idx % (2 * m);
            if (i == k) continue;
            const T f = S[i * SP + k];
            if (j < m) { if (j != k) S[i * SP + j] -= f * S[k * SP + j]; }
            else Si[i * SP + (j - m)] -= f * Si[k * SP + (j - m)];
        }
        __syncthreads();
        for (int i = tid; i < m; i += nth) if (i != k) S[i * SP + k] = T(0);
        __syncthreads();
    }
}

// One height of the cyclic reduction in every slab.
// grid = (node index a at this height, column chunk, slab t); block = TB_THREADS.
// SPD kinds: L L^T = S, Z = L^{-1} B; stored Linv, Z.  Indefinite kind: S^{-1} by pivoted
// Gauss-Jordan, W = S^{-1} B; stored S^{-1}, B (in the Z arrays) and W.  In both cases the
// condensed rows are R_merged = R_others - B^T S^{-1} B (= Z^T Z in the SPD form).
template <typename T, bool INDEF>
__global__ void __launch_bounds__(TB_THREADS) tree_factor_kernel(TreeArgs<T> A, int k) {
    __shared__ T S[MAXM * SP2];        // S (stride SP); indefinite kind: then W (stride SP2)
    __shared__ T Li[MAXM * SP];
    __shared__ T Bt[MAXM * SP2];       // B; SPD kind: then Z = Li B in place
    const int tid = threadIdx.x, nth = blockDim.x;
    const int t = blockIdx.z;
    const int c = (2 * blockIdx.x + 1) << k;
    const int s = A.s, m = A.m;
    if (c > s) return;
    const int lo = c - (1 << k) + 1;
    const int hi = min(s, c + (1 << k) - 1);
    const int w = hi - lo + 1;
    const int ncols = 2 * w;
    const int q0 = blockIdx.y * TB_THREADS;
    if (blockIdx.y > 0 && q0 >= ncols) return;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = tree_right_height(s, c, k);
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    const int x0 = t * A.b + 1;
    const int np1 = A.n + 1;
    const double* DGr = A.DG + (int64_t)c * np1;
    const double* AXr = A.AX + (int64_t)c * np1;
    const T* Ra = alpha ? A.rtb(t, alpha) : nullptr;
    const T* Rb = beta ? A.rtb(t, beta) : nullptr;
    const int m2 = 2 * m;

    // S = D_c + R_alpha[bot,bot] + R_beta[top,top];  B = [top | bot] couplings
    for (int idx = tid; idx < m * m; idx += nth) {
        const int i = idx / m, j = idx % m;
        double v = 0.0;
        if (i == j) v = DGr[x0 + i];
        else if (j == i + 1) v = -AXr[x0 + i];
        else if (j == i - 1) v = -AXr[x0 + j];
        T tv = (T)v;
        if (Ra) tv += Ra[(m + i) * m2 + (m + j)];
        if (Rb) tv += Rb[i * m2 + j];
        S[i * SP + j] = tv;
    }
    for (int idx = tid; idx < m * m2; idx += nth) {
        const int i = idx / m2, j = idx % m2;
        T v = T(0);
        if (j < m) {
            if (Ra) v = Ra[(m + i) * m2 + j];                       // alpha's bot row x its top column
            else if (i == j && c - 1 >= 1) v = (T)(-A.AY[(int64_t)(c - 1) * np1 + x0 + i]);
        } else {
            const int jj = j - m;
            if (Rb) v = Rb[i * m2 + m + jj];                        // beta's top row x its bot column
            else if (i == jj && c + 1 <= s) v = (T)(-A.AY[(int64_t)c * np1 + x0 + i]);
        }
        Bt[i * SP2 + j] = v;
    }
    __syncthreads();
    T* Wt = S;
    if (INDEF) {
        gj_inv_small<T>(S, Li, m, A.status);                        // Li = S^{-1}
        for (int idx = tid; idx < m * m2; idx += nth) {             // W = S^{-1} B (into S's buffer)
            const int i = idx / m2, j = idx % m2;
            T acc = T(0);
            for (int l = 0; l < m; ++l) acc += Li[i * SP + l] * Bt[l * SP2 + j];
            Wt[i * SP2 + j] = acc;
        }
    } else {
        chol_inv_small<T>(S, Li, m, A.status);
        // Z = Li B, in place; a thread owns a column, rows from the bottom (Li is lower triangular)
        for (int j = tid; j < m2; j += nth)
            for (int i = m - 1; i >= 0; --i) {
                T acc = T(0);
                for (int l = 0; l <= i; ++l) acc += Li[i * SP + l] * Bt[l * SP2 + j];
                Bt[i * SP2 + j] = acc;
            }
    }
    __syncthreads();
    const T* Zl = Bt;                  // left factor of the update: Z (SPD) or B (indefinite)
    const T* Zr = INDEF ? Wt : Bt;     // right factor: Z (SPD) or W (indefinite)
    if (blockIdx.y == 0) {
        T* Lg = A.linv(t, c);
        for (int idx = tid; idx < m * m; idx += nth) Lg[idx] = Li[(idx / m) * SP + idx % m];
        T* Zg = A.ztb(t, c);
        for (int idx = tid; idx < m * m2; idx += nth) Zg[idx] = Bt[(idx / m2) * SP2 + idx % m2];
        if (INDEF) {
            T* Wg = A.wtb(t, c);
            for (int idx = tid; idx < m * m2; idx += nth) Wg[idx] = Wt[(idx / m2) * SP2 + idx % m2];
        }
        T* Rg = A.rtb(t, c);
        for (int idx = tid; idx < m2 * m2; idx += nth) {
            const int a = idx / m2, bcol = idx % m2;
            T v = T(0);
            for (int l = 0; l < m; ++l) v -= Zl[l * SP2 + a] * Zr[l * SP2 + bcol];
            if (a < m && bcol < m && Ra) v += Ra[a * m2 + bcol];                     // alpha top x top
            if (a >= m && bcol >= m && Rb) v += Rb[a * m2 + bcol];                   // beta bot x bot
            Rg[idx] = v;
        }
    }
    // interface columns of the segment: one thread per column
    const int q = q0 + tid;
    if (q < ncols) {
        const int side = q / w;
        const int j = lo + q % w;
        const int rr = j - 1;
        const int sp = A.s_pad;
        T bvec[MAXM];
#pragma unroll
        for (int i = 0; i < MAXM; ++i) bvec[i] = T(0);
        if (j < c) {
            const T* src = A.ri(t, k - 1, 1, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) bvec[i] = src[(int64_t)i * sp];
        } else if (j == c) {
            if (side == 0) {
                if (t >= 1) bvec[0] = (T)(-AXr[x0 - 1]);
            } else {
                if (t <= A.NS - 2) {
#pragma unroll
                    for (int i = 0; i < MAXM; ++i) if (i == m - 1) bvec[i] = (T)(-AXr[x0 + m - 1]);
                }
            }
        } else {
            const T* src = A.ri(t, kb, 0, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) bvec[i] = src[(int64_t)i * sp];
        }
        T z[MAXM];                     // SPD: z = Li b; indefinite: w = S^{-1} b
#pragma unroll
        for (int i = 0; i < MAXM; ++i) {
            T acc = T(0);
#pragma unroll
            for (int l = 0; l < MAXM; ++l)
                if ((INDEF || l <= i) && l < m && i < m) acc += Li[i * SP + l] * bvec[l];
            z[i] = acc;
        }
        T* zd = A.zi(t, k, side) + rr;
        if (INDEF) {
            T* wd = A.wi(t, k, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i)
                if (i < m) {
                    zd[(int64_t)i * sp] = bvec[i];
                    wd[(int64_t)i * sp] = z[i];
                }
        } else {
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) zd[(int64_t)i * sp] = z[i];
        }
        // condensed top/bot rows for this interface column: R - Zl^T z  (Zl = Z or B)
        const T* rta = (j < c) ? A.ri(t, k - 1, 0, side) + rr : nullptr;
        const T* rbb = (j > c) ? A.ri(t, kb, 1, side) + rr : nullptr;
        T* rtd = A.ri(t, k, 0, side) + rr;
        T* rbd = A.ri(t, k, 1, side) + rr;
        for (int a = 0; a < m; ++a) {
            T vt = rta ? rta[(int64_t)a * sp] : T(0);
            T vb = rbb ? rbb[(int64_t)a * sp] : T(0);
#pragma unroll
            for (int i = 0; i < MAXM; ++i)
                if (i < m) {
                    vt -= Zl[i * SP2 + a] * z[i];
                    vb -= Zl[i * SP2 + m + a] * z[i];
                }
            rtd[(int64_t)a * sp] = vt;
            rbd[(int64_t)a * sp] = vb;
        }
    }
}

// One height of the cyclic reduction for the nonsymmetric kind (the same elimination as the
// indefinite kind with both orientations of every coupling kept).  Node c's separator block S,
// its row couplings B (separator rows x {top, bot, interface} columns) and column couplings C
// ({top, bot, interface} rows x separator columns) give
//   R_merged = R_others - C S^{-1} B,
// with S^{-1} from pivoted Gauss-Jordan.  Stored for A: S^{-1}, C^T, W = S^{-1} B; for A^T (whose
// separator block is S^T, row couplings C^T, column couplings B^T): S^{-T}, B, V = S^{-T} C^T.
// The condensed couplings are kept in both orientations: RI (top/bot rows x interface columns)
// and RIc (interface rows x top/bot columns).  grid = (node, column chunk, slab), as above.
template <typename T>
__global__ void __launch_bounds__(TB_THREADS) tree_factor_ns_kernel(TreeArgs<T> A, int k) {
    __shared__ T S[MAXM * SP2];        // S (stride SP), then W = S^{-1} B (stride SP2)
    __shared__ T Li[MAXM * SP];        // S^{-1}
    __shared__ T Bt[MAXM * SP2];       // B, then C^T
    const int tid = threadIdx.x, nth = blockDim.x;
    const int t = blockIdx.z;
    const int c = (2 * blockIdx.x + 1) << k;
    const int s = A.s, m = A.m;
    if (c > s) return;
    const int lo = c - (1 << k) + 1;
    const int hi = min(s, c + (1 << k) - 1);
    const int w = hi - lo + 1;
    const int ncols = 2 * w;
    const int q0 = blockIdx.y * TB_THREADS;
    if (blockIdx.y > 0 && q0 >= ncols) return;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = tree_right_height(s, c, k);
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    const int x0 = t * A.b + 1;
    const int np1 = A.n + 1;
    const double* DGr = A.DG + (int64_t)c * np1;
    const double* AXr = A.AX + (int64_t)c * np1;       // -h^2 A[(x,c),(x+1,c)]
    const double* AXTr = A.AXT + (int64_t)c * np1;     // -h^2 A[(x+1,c),(x,c)]
    const T* Ra = alpha ? A.rtb(t, alpha) : nullptr;   // alpha's rows/cols: top 0..m-1, bot m..2m-1
    const T* Rb = beta ? A.rtb(t, beta) : nullptr;
    const int m2 = 2 * m;

    // S = D_c + R_alpha[bot,bot] + R_beta[top,top];  B = couplings of row c to [top | bot]
    for (int idx = tid; idx < m * m; idx += nth) {
        const int i = idx / m, j = idx % m;
        double v = 0.0;
        if (i == j) v = DGr[x0 + i];
        else if (j == i + 1) v = -AXr[x0 + i];
        else if (j == i - 1) v = -AXTr[x0 + j];
        T tv = (T)v;
        if (Ra) tv += Ra[(m + i) * m2 + (m + j)];
        if (Rb) tv += Rb[i * m2 + j];
        S[i * SP + j] = tv;
    }
    for (int idx = tid; idx < m * m2; idx += nth) {
        const int i = idx / m2, j = idx % m2;
        T v = T(0);
        if (j < m) {
            if (Ra) v = Ra[(m + i) * m2 + j];                       // R_alpha[bot i][top j]
            else if (i == j && c - 1 >= 1) v = (T)(-A.AYT[(int64_t)(c - 1) * np1 + x0 + i]);
        } else {
            const int jj = j - m;
            if (Rb) v = Rb[i * m2 + m + jj];                        // R_beta[top i][bot jj]
            else if (i == jj && c + 1 <= s) v = (T)(-A.AY[(int64_t)c * np1 + x0 + i]);
        }
        Bt[i * SP2 + j] = v;
    }
    __syncthreads();
    gj_inv_small<T>(S, Li, m, A.status);                            // Li = S^{-1}
    T* Wt = S;
    for (int idx = tid; idx < m * m2; idx += nth) {                 // W = S^{-1} B (into S's buffer)
        const int i = idx / m2, j = idx % m2;
        T acc = T(0);
        for (int l = 0; l < m; ++l) acc += Li[i * SP + l] * Bt[l * SP2 + j];
        Wt[i * SP2 + j] = acc;
    }
    __syncthreads();
    if (blockIdx.y == 0) {
        T* Lg = A.linv(t, c);
        T* LTg = A.per_node(A.LinvT, t, c, m * m);
        for (int idx = tid; idx < m * m; idx += nth) {
            const int i = idx / m, j = idx % m;
            Lg[idx] = Li[i * SP + j];
            LTg[idx] = Li[j * SP + i];
        }
        T* Bg = A.per_node(A.ZtbT, t, c, m * m2);
        T* Wg = A.wtb(t, c);
        for (int idx = tid; idx < m * m2; idx += nth) {
            Bg[idx] = Bt[(idx / m2) * SP2 + idx % m2];
            Wg[idx] = Wt[(idx / m2) * SP2 + idx % m2];
        }
    }
    __syncthreads();
    // C^T: Ct[i][j] = coupling of top/bot node j into separator node i
    for (int idx = tid; idx < m * m2; idx += nth) {
        const int i = idx / m2, j = idx % m2;
        T v = T(0);
        if (j < m) {
            if (Ra) v = Ra[j * m2 + m + i];                         // R_alpha[top j][bot i]
            else if (i == j && c - 1 >= 1) v = (T)(-A.AY[(int64_t)(c - 1) * np1 + x0 + i]);
        } else {
            const int jj = j - m;
            if (Rb) v = Rb[(m + jj) * m2 + i];                      // R_beta[bot jj][top i]
            else if (i == jj && c + 1 <= s) v = (T)(-A.AYT[(int64_t)c * np1 + x0 + i]);
        }
        Bt[i * SP2 + j] = v;
    }
    __syncthreads();
    const T* Ct = Bt;
    if (blockIdx.y == 0) {
        T* Cg = A.ztb(t, c);
        T* Vg = A.per_node(A.WtbT, t, c, m * m2);
        for (int idx = tid; idx < m * m2; idx += nth) {
            const int i = idx / m2, j = idx % m2;
            Cg[idx] = Ct[i * SP2 + j];
            T acc = T(0);                                           // V = S^{-T} C^T
            for (int l = 0; l < m; ++l) acc += Li[l * SP + i] * Ct[l * SP2 + j];
            Vg[idx] = acc;
        }
        T* Rg = A.rtb(t, c);
        for (int idx = tid; idx < m2 * m2; idx += nth) {
            const int a = idx / m2, bcol = idx % m2;
            T v = T(0);
            for (int l = 0; l < m; ++l) v -= Ct[l * SP2 + a] * Wt[l * SP2 + bcol];
            if (a < m && bcol < m && Ra) v += Ra[a * m2 + bcol];                     // alpha top x top
            if (a >= m && bcol >= m && Rb) v += Rb[a * m2 + bcol];                   // beta bot x bot
            Rg[idx] = v;
        }
    }
    // interface columns of the segment: one thread per column
    const int q = q0 + tid;
    if (q < ncols) {
        const int side = q / w;
        const int j = lo + q % w;
        const int rr = j - 1;
        const int sp = A.s_pad;
        T vec[MAXM], z[MAXM];
        // (1) b = coupling of the separator rows to interface node j; W column z = S^{-1} b
#pragma unroll
        for (int i = 0; i < MAXM; ++i) vec[i] = T(0);
        if (j < c) {
            const T* src = A.ri(t, k - 1, 1, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) vec[i] = src[(int64_t)i * sp];
        } else if (j == c) {
            if (side == 0) {
                if (t >= 1) vec[0] = (T)(-AXTr[x0 - 1]);              // A[(x0,c),(x0-1,c)]
            } else {
                if (t <= A.NS - 2) {
#pragma unroll
                    for (int i = 0; i < MAXM; ++i) if (i == m - 1) vec[i] = (T)(-AXr[x0 + m - 1]);
                }
            }
        } else {
            const T* src = A.ri(t, kb, 0, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) vec[i] = src[(int64_t)i * sp];
        }
#pragma unroll
        for (int i = 0; i < MAXM; ++i) {
            T acc = T(0);
#pragma unroll
            for (int l = 0; l < MAXM; ++l)
                if (l < m && i < m) acc += Li[i * SP + l] * vec[l];
            z[i] = acc;
        }
        {
            T* bd = A.per_height(A.ZIT, t, k, side) + rr;
            T* wd = A.per_height(A.WI, t, k, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i)
                if (i < m) {
                    bd[(int64_t)i * sp] = vec[i];
                    wd[(int64_t)i * sp] = z[i];
                }
        }
        // condensed top/bot rows x this column: RI = R_child - C[tb, sep] z
        {
            const T* rta = (j < c) ? A.ri(t, k - 1, 0, side) + rr : nullptr;
            const T* rbb = (j > c) ? A.ri(t, kb, 1, side) + rr : nullptr;
            T* rtd = A.ri(t, k, 0, side) + rr;
            T* rbd = A.ri(t, k, 1, side) + rr;
            for (int a = 0; a < m; ++a) {
                T vt = rta ? rta[(int64_t)a * sp] : T(0);
                T vb = rbb ? rbb[(int64_t)a * sp] : T(0);
#pragma unroll
                for (int i = 0; i < MAXM; ++i)
                    if (i < m) {
                        vt -= Ct[i * SP2 + a] * z[i];
                        vb -= Ct[i * SP2 + m + a] * z[i];
                    }
                rtd[(int64_t)a * sp] = vt;
                rbd[(int64_t)a * sp] = vb;
            }
        }
        // (2) c = coupling of interface node j into the separator columns; V column z = S^{-T} c
#pragma unroll
        for (int i = 0; i < MAXM; ++i) vec[i] = T(0);
        if (j < c) {
            const T* src = A.ric(t, k - 1, 1, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) vec[i] = src[(int64_t)i * sp];
        } else if (j == c) {
            if (side == 0) {
                if (t >= 1) vec[0] = (T)(-AXr[x0 - 1]);               // A[(x0-1,c),(x0,c)]
            } else {
                if (t <= A.NS - 2) {
#pragma unroll
                    for (int i = 0; i < MAXM; ++i) if (i == m - 1) vec[i] = (T)(-AXTr[x0 + m - 1]);
                }
            }
        } else {
            const T* src = A.ric(t, kb, 0, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i) if (i < m) vec[i] = src[(int64_t)i * sp];
        }
#pragma unroll
        for (int i = 0; i < MAXM; ++i) {
            T acc = T(0);
#pragma unroll
            for (int l = 0; l < MAXM; ++l)
                if (l < m && i < m) acc += Li[l * SP + i] * vec[l];
            z[i] = acc;
        }
        {
            T* cd = A.zi(t, k, side) + rr;
            T* vd = A.per_height(A.WIT, t, k, side) + rr;
#pragma unroll
            for (int i = 0; i < MAXM; ++i)
                if (i < m) {
                    cd[(int64_t)i * sp] = vec[i];
                    vd[(int64_t)i * sp] = z[i];
                }
        }
        // condensed interface row x top/bot columns: RIc = R_child - c^T W[:, tb]
        {
            const T* rta = (j < c) ? A.ric(t, k - 1, 0, side) + rr : nullptr;
            const T* rbb = (j > c) ? A.ric(t, kb, 1, side) + rr : nullptr;
            T* rtd = A.ric(t, k, 0, side) + rr;
            T* rbd = A.ric(t, k, 1, side) + rr;
            for (int a = 0; a < m; ++a) {
                T vt = rta ? rta[(int64_t)a * sp] : T(0);
                T vb = rbb ? rbb[(int64_t)a * sp] : T(0);
#pragma unroll
                for (int i = 0; i < MAXM; ++i)
                    if (i < m) {
                        vt -= vec[i] * Wt[i * SP2 + a];
                        vb -= vec[i] * Wt[i * SP2 + m + a];
                    }
                rtd[(int64_t)a * sp] = vt;
                rbd[(int64_t)a * sp] = vb;
            }
        }
    }
}

// ------------------------------------------------------------------ solve phases
template <typename T>
struct SolveArgs {
    TreeArgs<T> tr;
    int K;            // right-hand sides in this call (<= kcap)
    int kcap;         // stride of the right-hand-side index
    T* Yv;            // [NS][s+1][m][kcap]
    T* Gtb;           // [NS][s+1][2][m][kcap]
    T* Xs;            // [NS][s+1][m][kcap]
    T* Fi;            // [NS][2][s_pad][kcap]
    T* X;             // [NI][kcap][s_pad]  right-hand-side major
    __device__ int64_t nodeoff(int t, int c) const { return (int64_t)t * (tr.s + 1) + c; }
    __device__ T* yv(int t, int c) const { return Yv + nodeoff(t, c) * tr.m * kcap; }
    __device__ T* gtb(int t, int c, int tb) const { return Gtb + (nodeoff(t, c) * 2 + tb) * tr.m * kcap; }
    __device__ T* xs(int t, int c) const { return Xs + nodeoff(t, c) * tr.m * kcap; }
    __device__ T* fi(int t, int side) const { return Fi + ((int64_t)t * 2 + side) * tr.s_pad * kcap; }
    __device__ T* xi(int q) const { return X + (int64_t)q * tr.s_pad * kcap; }   // [kcap][s_pad]
};

constexpr int KMAX = 64;   // right-hand sides handled per launch
constexpr int LP = 36;     // smem row stride of the 32-row blocks read 4 at a time (16-byte aligned)
constexpr int KP = KMAX + 4;   // smem row stride of the m x K blocks: 16-byte aligned, rows 4 banks apart

// Lane -> (row i, right-hand side r) inside a warp tile of 8 rows x 4 right-hand sides, for the
// copies between a [row][r] smem block of stride KP and global memory contiguous in the row
// index: the smem words (KP i + r) of a warp (a half-warp for double) fall in distinct banks,
// and the global side touches four (double: eight) 32-byte segments per warp.
template <typename T>
__device__ inline void lane_rows_rhs(int lane, int& i, int& r) {
    if (sizeof(T) == 8) { i = (lane & 3) | ((lane >> 4) << 2); r = (lane >> 2) & 3; }
    else { i = lane & 7; r = lane >> 3; }
}

// four consecutive smem values (16-byte aligned): one 128-bit store for float, two for double
__device__ inline void sts4(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ inline void sts4(double* p, const double v[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// four consecutive smem values (16-byte aligned): one 128-bit load for float, two for double
__device__ inline void lds4(const float* p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ inline void lds4(const double* p, double v[4]) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Up pass of one height: y = Li (f_c + G_alpha[bot] + G_beta[top]); condensed top/bot load;
// interface load Fi -= Z_I^T y.  grid = (node, chunk, slab).  The m x K products use 4 x 4
// register blocks: thread (tA, tB) owns rows 4tA..4tA+3 and right-hand sides 4tB..4tB+3.
template <typename T>
__global__ void __launch_bounds__(TB_THREADS, sizeof(T) == 8 ? 5 : 8) tree_up_kernel(SolveArgs<T> P, int k, const double* F,
                                                             double fscale, int r0) {
    constexpr int ZP = 2 * MAXM + 4;   // Zt row stride: top half at 0, bottom half at MAXM
    __shared__ __align__(16) T Li[MAXM * LP];      // Li[l][i] = (L^{-1})[i][l], zero outside m x m
    __shared__ __align__(16) T Zt[MAXM * ZP];      // Zt[i][tb MAXM + a] = Z[i][tb m + a], zero for a >= m
    __shared__ __align__(16) T y[MAXM * KP];
    // 32 interface columns of Z_I, staged per pass; Zt is no longer read by then
    T* const zs = Zt;
    static_assert(ZP >= LP, "staging area must fit in Zt");
    const TreeArgs<T>& A = P.tr;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int tA = tid >> 4, tB = tid & 15;
    const int t = blockIdx.z;
    const int c = (2 * blockIdx.x + 1) << k;
    const int s = A.s, m = A.m, K = P.K, kc = P.kcap;
    if (c > s) return;
    const int lo = c - (1 << k) + 1;
    const int hi = min(s, c + (1 << k) - 1);
    const int w = hi - lo + 1;
    const int ncols = 2 * w;
    const int q0 = blockIdx.y * TB_THREADS;
    if (blockIdx.y > 0 && q0 >= ncols) return;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = tree_right_height(s, c, k);
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    const int x0 = t * A.b + 1;
    const int m2 = 2 * m;
    const T* Lg = A.linv(t, c);
    const T* Zg = A.ztb(t, c);
    // Zt: rows by warp, columns by lane.  Li transposed through tiles of JB columns x 32/JB rows
    // per warp (jl fast): smem words (LP l + i) of a wavefront fall in distinct banks.  Each
    // group of loads is issued into registers before its stores.
    constexpr int NW = TB_THREADS / 32;
    const int lane = tid & 31, warp = tid >> 5;
    {
        constexpr int JB = sizeof(T) == 8 ? 4 : 8;
        constexpr int LIT = (MAXM / JB) * (MAXM / (32 / JB)) / NW;
        const int jl = lane % JB, il = lane / JB;
        T z0[MAXM / NW], z1[MAXM / NW], lr[LIT];
#pragma unroll
        for (int it = 0; it < MAXM / NW; ++it) {
            const int i = warp + NW * it;
            const bool ok = i < m && lane < m;
            z0[it] = ok ? Zg[i * m2 + lane] : T(0);
            z1[it] = ok ? Zg[i * m2 + m + lane] : T(0);
        }
#pragma unroll
        for (int it = 0; it < LIT; ++it) {
            const int wb = warp + NW * it;
            const int l = JB * (wb % (MAXM / JB)) + jl, i = (32 / JB) * (wb / (MAXM / JB)) + il;
            lr[it] = (i < m && l < m) ? Lg[i * m + l] : T(0);
        }
#pragma unroll
        for (int it = 0; it < MAXM / NW; ++it) {
            const int i = warp + NW * it;
            Zt[i * ZP + lane] = z0[it];
            Zt[i * ZP + MAXM + lane] = z1[it];
        }
#pragma unroll
        for (int it = 0; it < LIT; ++it) {
            const int wb = warp + NW * it;
            const int l = JB * (wb % (MAXM / JB)) + jl, i = (32 / JB) * (wb / (MAXM / JB)) + il;
            Li[l * LP + i] = lr[it];
        }
    }
    const int64_t N = (int64_t)s * s;
    {
        constexpr int YIT = (MAXM / 8) * (KMAX / 4) / NW;
        int il, rl;
        lane_rows_rhs<T>(lane, il, rl);
        T g[YIT];
#pragma unroll
        for (int it = 0; it < YIT; ++it) {
            const int wb = warp + NW * it;
            const int i = 8 * (wb % (MAXM / 8)) + il, r = 4 * (wb / (MAXM / 8)) + rl;
            g[it] = (i < m && r < K)
                        ? (T)F[(int64_t)(r0 + r) * N + (int64_t)(c - 1) * s + (x0 - 1 + i)] * (T)fscale
                        : T(0);
        }
        if (alpha) {
            const T* ga = P.gtb(t, alpha, 1);
#pragma unroll
            for (int it = 0; it < YIT; ++it) {
                const int wb = warp + NW * it;
                const int i = 8 * (wb % (MAXM / 8)) + il, r = 4 * (wb / (MAXM / 8)) + rl;
                if (i < m && r < K) g[it] += ga[i * kc + r];
            }
        }
        if (beta) {
            const T* gb = P.gtb(t, beta, 0);
#pragma unroll
            for (int it = 0; it < YIT; ++it) {
                const int wb = warp + NW * it;
                const int i = 8 * (wb % (MAXM / 8)) + il, r = 4 * (wb / (MAXM / 8)) + rl;
                if (i < m && r < K) g[it] += gb[i * kc + r];
            }
        }
#pragma unroll
        for (int it = 0; it < YIT; ++it) {
            const int wb = warp + NW * it;
            y[(8 * (wb % (MAXM / 8)) + il) * KP + 4 * (wb / (MAXM / 8)) + rl] = g[it];
        }
    }
    __syncthreads();
    // y = Li g
    {
        T acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
        for (int l = 0; l < m; ++l) {
            T gv[4], lv[4];
            lds4(y + l * KP + 4 * tB, gv);
            lds4(Li + l * LP + 4 * tA, lv);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += lv[q] * gv[p];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) sts4(y + (4 * tA + q) * KP + 4 * tB, acc[q]);
    }
    __syncthreads();
    if (blockIdx.y == 0) {
        T* yd = P.yv(t, c);
        for (int i = tid >> 6; i < m; i += nth >> 6) {
            const int r = tid & 63;
            if (r < K) yd[i * kc + r] = y[i * KP + r];
        }
        // condensed top / bottom loads: G_tb[a][r] = G_child[a][r] - sum_i Z[i][tb*m + a] y[i][r]
        for (int tb = 0; tb < 2; ++tb) {
            const int child = tb == 0 ? alpha : beta;
            T acc[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
            for (int i = 0; i < m; ++i) {
                T yv[4], zv[4];
                lds4(y + i * KP + 4 * tB, yv);
                lds4(Zt + i * ZP + tb * MAXM + 4 * tA, zv);
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int p = 0; p < 4; ++p) acc[q][p] += zv[q] * yv[p];
            }
            const T* gc = child ? P.gtb(t, child, tb) : nullptr;
            T* gd = P.gtb(t, c, tb);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int a = 4 * tA + q;
                if (a >= m) continue;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int r = 4 * tB + p;
                    if (r < K) gd[a * kc + r] = (gc ? gc[a * kc + r] : T(0)) - acc[q][p];
                }
            }
        }
    }
    // interface load: Fi[side][rr][r] -= sum_i Z_I[i][rr] y[i][r]
    const int qend = min(ncols, q0 + TB_THREADS);
    if (qend - q0 <= 16) {
        // few columns (low heights): thread = (column, group of RB right-hand sides)
        const int nq = qend - q0;
        const int RB = nq <= 2 ? 1 : (nq <= 4 ? 2 : (nq <= 8 ? 4 : 8));
        const int groups = KMAX / RB;
        const int qq = tid / groups, r0b = (tid % groups) * RB;
        if (qq < nq && r0b < K) {
            const int col = q0 + qq;
            const int sd = col / w, rr = lo + col % w - 1;
            const T* zcol = A.zi(t, k, sd) + rr;
            T acc[8], zv[MAXM];
#pragma unroll
            for (int p = 0; p < 8; ++p) acc[p] = T(0);
#pragma unroll
            for (int i = 0; i < MAXM; ++i) zv[i] = i < m ? zcol[(int64_t)i * A.s_pad] : T(0);
#pragma unroll
            for (int i = 0; i < MAXM; ++i) {
                if (i >= m) break;
#pragma unroll
                for (int p = 0; p < 8; ++p)
                    if (p < RB) acc[p] += zv[i] * y[i * KP + r0b + p];
            }
            T* fo = P.fi(t, sd) + (int64_t)rr * kc;
#pragma unroll
            for (int p = 0; p < 8; ++p)
                if (p < RB && r0b + p < K) fo[r0b + p] -= acc[p];
        }
        return;
    }
    for (int qa = q0; qa < qend; qa += 32) {
        int sd[4], rr[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int qq = qa + 4 * tA + q;
            ok[q] = qq < qend;
            sd[q] = ok[q] ? qq / w : 0;
            rr[q] = ok[q] ? lo + qq % w - 1 : 0;
        }
        // stage Z_I[i][columns qa .. qa+31] (rows by warp, columns by lane: coalesced)
        T zr[MAXM / NW];
        {
            const int qq = qa + lane;
            const int sdq = qq >= w, rq = lo + (sdq ? qq - w : qq) - 1;
            const T* zsrc = A.zi(t, k, sdq) + rq;
#pragma unroll
            for (int it = 0; it < MAXM / NW; ++it) {
                const int i = warp + NW * it;
                zr[it] = (i < m && qq < qend) ? zsrc[(int64_t)i * A.s_pad] : T(0);
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < MAXM / NW; ++it) zs[(warp + NW * it) * LP + lane] = zr[it];
        __syncthreads();
        T acc[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
        for (int i = 0; i < m; ++i) {
            T yv[4], zv[4];
            lds4(y + i * KP + 4 * tB, yv);
            lds4(zs + i * LP + 4 * tA, zv);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += zv[q] * yv[p];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!ok[q]) continue;
            T* fo = P.fi(t, sd[q]) + (int64_t)rr[q] * kc;
#pragma unroll
            for (int p = 0; p < 4; ++p)
                if (4 * tB + p < K) fo[4 * tB + p] -= acc[q][p];
        }
    }
}

// Down pass of one height: x_c = Li^T (y - Z_top x_top - Z_bot x_bot - Z_I u_I).
// grid = (node, chunk, slab).  A node's 2w interface columns are split into chunks of DCW; each
// CTA reduces its chunk (chunk 0 also the 2m top/bottom columns) into a partial V (m x K) held
// in 4 x 4 register blocks.  Nodes with one chunk finish in place; otherwise the partials go to
// ws and the last CTA of the node (ticket) adds them in chunk order and finishes the node.
constexpr int DCW = 256;      // largest chunk; heights with few nodes use smaller chunks (down_chunk)
constexpr int DCW_MIN = 32;

// Interface columns per CTA of the down pass at a height with `nodes` nodes of 2 wmax columns:
// enough CTAs to fill the GPU (about 4 per SM) without chunks narrower than DCW_MIN.
inline int down_chunk(int nodes, int wmax) {
    int c = DCW;
    while (c > DCW_MIN && (int64_t)nodes * ((2 * wmax + c - 1) / c) < 4 * 152) c /= 2;
    return c;
}
template <typename T, bool INDEF>
__global__ void __launch_bounds__(TB_THREADS, sizeof(T) == 8 ? 5 : 8) tree_down_kernel(SolveArgs<T> P, int k, double* U,
                                                               int accumulate, int r0, T* ws,
                                                               unsigned* tickets, int dcw) {
    constexpr int CJ = sizeof(T) == 8 ? 16 : 32;   // columns per smem stage
    constexpr int NW = TB_THREADS / 32;
    // Staging tiles of 32 elements per warp: lane (jl, il) with jl fast.  zc[jj][i] and uc[jj][r]
    // rows are LP (KP) words apart = 4 banks, so 8 columns x 4 rows (double: 4 x 8, 16 lanes
    // per wavefront) hit distinct banks while the global side reads 32-byte segments along the
    // column index.  Stages made only of top/bottom columns read x_top / x_bot, which are
    // contiguous in r, with r on the lanes instead.  Each thread issues all loads of a stage
    // into registers before the barrier that frees the smem tiles.
    constexpr int JB = sizeof(T) == 8 ? 4 : 8;
    constexpr int ZIT = (CJ / JB) * (MAXM / (32 / JB)) / NW;   // zc tiles per warp
    constexpr int UIT = (CJ / JB) * (KMAX / (32 / JB)) / NW;   // uc tiles per warp
    static_assert(UIT == (CJ / NW) * (KMAX / 32), "top/bottom staging covers the same tile count");
    __shared__ __align__(16) T Li[MAXM * LP];          // Li[l][i], zero for i >= m
    __shared__ __align__(16) T V[MAXM * KP];
    __shared__ __align__(16) T zc[CJ * LP];            // zc[jj][i]: column jj of the stage, rows i
    __shared__ __align__(16) T uc[CJ * KP];            // uc[jj][r]: column jj of the stage, rhs r
    __shared__ bool last;
    const TreeArgs<T>& A = P.tr;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int tA = tid >> 4, tB = tid & 15;
    const int t = blockIdx.z;
    const int c = (2 * blockIdx.x + 1) << k;
    const int s = A.s, m = A.m, K = P.K, kc = P.kcap;
    if (c > s) return;
    const int lo = c - (1 << k) + 1;
    const int hi = min(s, c + (1 << k) - 1);
    const int w = hi - lo + 1;
    const int nch = (2 * w + dcw - 1) / dcw;
    if ((int)blockIdx.y >= nch) return;
    const int qa = blockIdx.y * dcw, qb = min(2 * w, qa + dcw);
    const int x0 = t * A.b + 1;
    const int m2 = 2 * m;
    // acc accumulates -y + sum_j z_j u_j^T (y only in chunk 0), so that V = y - sum = -acc.
    // The y loads and the Li staging are issued first and overlap the first stage.
    T acc[4][4];
    if (blockIdx.y == 0) {
        const T* yv = P.yv(t, c);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int row = 4 * tA + q, r = 4 * tB + p;
                acc[q][p] = (row < m && r < K) ? -yv[row * kc + r] : T(0);
            }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
    }
    if (!INDEF) {
        const T* Lg = A.linv(t, c);
        T lr[MAXM / NW];
#pragma unroll
        for (int it = 0; it < MAXM / NW; ++it) {
            const int i = warp + NW * it;
            lr[it] = (i < m && lane < m) ? Lg[i * m + lane] : T(0);
        }
#pragma unroll
        for (int it = 0; it < MAXM / NW; ++it) Li[(warp + NW * it) * LP + lane] = lr[it];
    }
    const T* Zg = INDEF ? A.wtb(t, c) : A.ztb(t, c);    // SPD: Z; indefinite: W = S^{-1} B
    const T* xt = (lo - 1 >= 1) ? P.xs(t, lo - 1) : nullptr;
    const T* xb = (hi + 1 <= s) ? P.xs(t, hi + 1) : nullptr;
    // one list of columns: the 2m top/bot columns (chunk 0 only), then this chunk's interface
    // columns of the left (ic < w) and right side; staged CJ at a time
    const int ntb = blockIdx.y == 0 ? m2 : 0;
    const int ntot = ntb + (qb - qa);
    const T* ZIl = (t >= 1) ? (INDEF ? A.wi(t, k, 0) : A.zi(t, k, 0)) + (lo - 1) : nullptr;
    const T* ZIr = (t < A.NS - 1) ? (INDEF ? A.wi(t, k, 1) : A.zi(t, k, 1)) + (lo - 1) : nullptr;
    const T* Ul = (t >= 1) ? P.xi(t - 1) + (lo - 1) : nullptr;
    const T* Ur = (t < A.NS - 1) ? P.xi(t) + (lo - 1) : nullptr;
    const int jl = lane % JB, il = lane / JB;
    for (int v0 = 0; v0 < ntot; v0 += CJ) {
        const int nj = min(CJ, ntot - v0);
        T zr[ZIT], ur[UIT];
#pragma unroll
        for (int it = 0; it < ZIT; ++it) {
            const int wb = warp + NW * it;
            const int jj = JB * (wb % (CJ / JB)) + jl, i = (32 / JB) * (wb / (CJ / JB)) + il;
            const int col = v0 + jj;
            T z = T(0);
            if (jj < nj && i < m) {
                if (col < ntb) {
                    z = Zg[(int64_t)i * m2 + col];
                } else {
                    const int ic = qa + col - ntb;
                    const bool right = ic >= w;
                    const T* zs = right ? ZIr : ZIl;
                    if (zs) z = zs[(int64_t)i * A.s_pad + (right ? ic - w : ic)];
                }
            }
            zr[it] = z;
        }
        const bool tb_only = v0 + CJ <= ntb;
        if (tb_only) {
#pragma unroll
            for (int it = 0; it < UIT; ++it) {
                const int jj = warp + NW * (it / (KMAX / 32)), r = lane + 32 * (it % (KMAX / 32));
                const int col = v0 + jj;
                const T* xv = col < m ? xt : xb;
                ur[it] = (xv && r < K) ? xv[(col < m ? col : col - m) * kc + r] : T(0);
            }
        } else {
#pragma unroll
            for (int it = 0; it < UIT; ++it) {
                const int wb = warp + NW * it;
                const int jj = JB * (wb % (CJ / JB)) + jl, r = (32 / JB) * (wb / (CJ / JB)) + il;
                const int col = v0 + jj;
                T v = T(0);
                if (jj < nj && r < K) {
                    if (col < ntb) {
                        const T* xv = col < m ? xt : xb;
                        if (xv) v = xv[(col < m ? col : col - m) * kc + r];
                    } else {
                        const int ic = qa + col - ntb;
                        const bool right = ic >= w;
                        const T* us = right ? Ur : Ul;
                        if (us) v = us[(int64_t)r * A.s_pad + (right ? ic - w : ic)];
                    }
                }
                ur[it] = v;
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < ZIT; ++it) {
            const int wb = warp + NW * it;
            const int jj = JB * (wb % (CJ / JB)) + jl, i = (32 / JB) * (wb / (CJ / JB)) + il;
            zc[jj * LP + i] = zr[it];
        }
        if (tb_only) {
#pragma unroll
            for (int it = 0; it < UIT; ++it)
                uc[(warp + NW * (it / (KMAX / 32))) * KP + lane + 32 * (it % (KMAX / 32))] = ur[it];
        } else {
#pragma unroll
            for (int it = 0; it < UIT; ++it) {
                const int wb = warp + NW * it;
                const int jj = JB * (wb % (CJ / JB)) + jl, r = (32 / JB) * (wb / (CJ / JB)) + il;
                uc[jj * KP + r] = ur[it];
            }
        }
        __syncthreads();
        for (int jj = 0; jj < nj; ++jj) {
            T zv[4], uv[4];
            lds4(zc + jj * LP + 4 * tA, zv);
            lds4(uc + jj * KP + 4 * tB, uv);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += zv[q] * uv[p];
        }
    }
    if (nch > 1) {
        // partial of this chunk straight from the registers; the last CTA of the node adds the
        // partials in chunk order (deterministic), loading a thread's 16 elements together
        T* wsn = ws + ((int64_t)(t * gridDim.x + blockIdx.x) * nch) * MAXM * KMAX;
        T* wsc = wsn + (int64_t)blockIdx.y * MAXM * KMAX;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) wsc[(4 * tA + q) * KMAX + 4 * tB + p] = acc[q][p];
        __threadfence();
        __syncthreads();
        unsigned* tk = tickets + (int64_t)t * gridDim.x + blockIdx.x;
        if (tid == 0) last = atomicAdd(tk, 1u) == (unsigned)(nch - 1);
        __syncthreads();
        if (!last) return;
        __threadfence();
        constexpr int PER = MAXM * KMAX / TB_THREADS;
        T v[PER];
#pragma unroll
        for (int j = 0; j < PER; ++j) v[j] = T(0);
        for (int ch = 0; ch < nch; ++ch) {
            const T* src = wsn + (int64_t)ch * MAXM * KMAX + tid;
            T ld[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) ld[j] = __ldcg(src + j * TB_THREADS);
#pragma unroll
            for (int j = 0; j < PER; ++j) v[j] += ld[j];
        }
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int idx = tid + j * TB_THREADS;
            V[(idx / KMAX) * KP + idx % KMAX] = -v[j];
        }
        if (tid == 0) *tk = 0;
    } else {
        __syncthreads();   // zc / uc reads of the last stage are not affected; V is free
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const T nv[4] = {-acc[q][0], -acc[q][1], -acc[q][2], -acc[q][3]};
            sts4(V + (4 * tA + q) * KP + 4 * tB, nv);
        }
    }
    __syncthreads();
    // finish the node: V = y - sum; SPD: x = Li^T V, indefinite: x = V (y already holds S^{-1} g)
    if (!INDEF) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
        for (int l = 0; l < m; ++l) {                      // x[i] = sum_{l >= i} Li[l][i] V[l]
            T lv[4], vv[4];
            lds4(Li + l * LP + 4 * tA, lv);
            lds4(V + l * KP + 4 * tB, vv);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int p = 0; p < 4; ++p) acc[q][p] += lv[q] * vv[p];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) sts4(V + (4 * tA + q) * KP + 4 * tB, acc[q]);
        __syncthreads();
    }
    const int64_t N = (int64_t)s * s;
    if (k > 0) {                       // x of a height-0 row is read by no lower node
        T* xd = P.xs(t, c);
        for (int i = tid >> 6; i < m; i += TB_THREADS >> 6) {
            const int r = tid & 63;
            if (r < K) xd[i * kc + r] = V[i * KP + r];
        }
    }
    {
        int ul, rl;
        lane_rows_rhs<T>(lane, ul, rl);
        for (int wb = warp; wb < (MAXM / 8) * (KMAX / 4); wb += NW) {
            const int i = 8 * (wb % (MAXM / 8)) + ul, r = 4 * (wb / (MAXM / 8)) + rl;
            if (i < m && r < K) {
                const double v = (double)V[i * KP + r];
                double* up = U + (int64_t)(r0 + r) * N + (int64_t)(c - 1) * s + (x0 - 1 + i);
                if (accumulate) *up += v;
                else *up = v;
            }
        }
    }
}

// X[q][r][rr] = fscale f[r][rr][x_q] + Fi[q][R][rr][r] + Fi[q+1][L][rr][r]  (padding rows zero)
template <typename T>
__global__ void gather_ftilde_kernel(SolveArgs<T> P, const double* F, double fscale, int r0) {
    const TreeArgs<T>& A = P.tr;
    const int q = blockIdx.y;
    const int K = P.K, kc = P.kcap;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)A.s_pad * K) return;
    const int r = (int)(idx / A.s_pad), rr = (int)(idx % A.s_pad);
    T v = T(0);
    if (rr < A.s) {
        const int64_t N = (int64_t)A.s * A.s;
        const int xq = (q + 1) * A.b;
        v = (T)(fscale * F[(int64_t)(r0 + r) * N + (int64_t)rr * A.s + (xq - 1)]);
        v += P.fi(q, 1)[(int64_t)rr * kc + r] + P.fi(q + 1, 0)[(int64_t)rr * kc + r];
    }
    P.xi(q)[(int64_t)r * A.s_pad + rr] = v;
}

template <typename T>
__global__ void scatter_utilde_kernel(SolveArgs<T> P, double* U, int accumulate, int r0) {
    const TreeArgs<T>& A = P.tr;
    const int q = blockIdx.y;
    const int K = P.K, kc = P.kcap;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)A.s * K) return;
    const int rr = (int)(idx % A.s), r = (int)(idx / A.s);
    const int64_t N = (int64_t)A.s * A.s;
    const int xq = (q + 1) * A.b;
    double* up = U + (int64_t)(r0 + r) * N + (int64_t)rr * A.s + (xq - 1);
    const double v = (double)P.xi(q)[(int64_t)r * A.s_pad + rr];
    if (accumulate) *up += v;
    else *up = v;
}

// ftilde (FP64, [k][q][j]) <-> X (scalar, [q][j][r])
template <typename T>
__global__ void export_x_kernel(SolveArgs<T> P, double* out, double scale, int NI, int r0) {
    const TreeArgs<T>& A = P.tr;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)NI * A.s;
    if (idx >= per * P.K) return;
    const int r = (int)(idx / per);
    const int64_t rem = idx % per;
    const int q = (int)(rem / A.s), rr = (int)(rem % A.s);
    out[(int64_t)(r0 + r) * per + rem] = scale * (double)P.xi(q)[(int64_t)r * A.s_pad + rr];
}
template <typename T>
__global__ void import_x_kernel(SolveArgs<T> P, const double* in, int NI, int r0) {
    const TreeArgs<T>& A = P.tr;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)NI * A.s_pad;
    if (idx >= per * P.K) return;
    const int r = (int)(idx / per);
    const int64_t rem = idx % per;
    const int q = (int)(rem / A.s_pad), rr = (int)(rem % A.s_pad);
    P.xi(q)[(int64_t)r * A.s_pad + rr] =
        rr < A.s ? (T)in[(int64_t)(r0 + r) * NI * A.s + (int64_t)q * A.s + rr] : T(0);
}

template <typename T>
TreeArgs<T> make_tree_args(slab_handle* h) {
    TreeArgs<T> a{};
    a.s = h->td.s; a.s_pad = h->td.s_pad; a.m = h->td.m; a.H = h->td.H; a.NS = h->td.NS;
    a.b = h->b; a.n = h->n;
    a.AX = h->AX; a.AY = h->AY; a.DG = h->DG;
    a.Linv = (T*)h->tLinv; a.Ztb = (T*)h->tZtb; a.Rtb = (T*)h->tRtb; a.ZI = (T*)h->tZI; a.RI = (T*)h->tRI;
    a.Wtb = (T*)h->tWtb; a.WI = (T*)h->tWI;
    a.AXT = h->AXT; a.AYT = h->AYT;
    a.LinvT = (T*)h->tLinvT; a.ZtbT = (T*)h->tZtbT; a.WtbT = (T*)h->tWtbT;
    a.ZIT = (T*)h->tZIT; a.WIT = (T*)h->tWIT; a.RIc = (T*)h->tRIc;
    a.status = h->dstatus;
    if (h->transposed && h->kind == SLAB_CONVECTION) {
        // A^T's elimination: separator inverse S^{-T}, couplings into the separators B (was C^T),
        // the back-substitution columns V = S^{-T} C^T (was W = S^{-1} B)
        a.Linv = a.LinvT; a.Ztb = a.ZtbT; a.ZI = a.ZIT; a.Wtb = a.WtbT; a.WI = a.WIT;
    }
    return a;
}

template <typename T>
SolveArgs<T> make_solve_args(slab_handle* h, int K) {
    SolveArgs<T> p;
    p.tr = make_tree_args<T>(h);
    p.K = K; p.kcap = h->kcap;
    p.Yv = (T*)h->wYv; p.Gtb = (T*)h->wGtb; p.Xs = (T*)h->wXs; p.Fi = (T*)h->wFi; p.X = (T*)h->wX;
    return p;
}

inline int chunks_at(int s, int k) {
    const int wmax = min(s, (1 << (k + 1)) - 1);
    return (2 * wmax + TB_THREADS - 1) / TB_THREADS;
}

}  // namespace

template <typename T>
slab_status tree_factor(slab_handle* h) {
    TreeArgs<T> a = make_tree_args<T>(h);
    const TreeDims& d = h->td;
    const bool indef = h->kind == SLAB_HELMHOLTZ;
    const bool nonsym = h->kind == SLAB_CONVECTION;
    for (int k = 0; k < d.H; ++k) {
        const int cnt = tree_nodes_at(d.s, k);
        if (!cnt) continue;
        dim3 grid(cnt, chunks_at(d.s, k), d.NS);
        SLAB_PROF(h, KC_TREE_FACTOR);
        if (nonsym) tree_factor_ns_kernel<T><<<grid, TB_THREADS, 0, h->stream>>>(a, k);
        else if (indef) tree_factor_kernel<T, true><<<grid, TB_THREADS, 0, h->stream>>>(a, k);
        else tree_factor_kernel<T, false><<<grid, TB_THREADS, 0, h->stream>>>(a, k);
        SLAB_CK_LAUNCH(h);
        if (slab_debug() && slab_debug_status(h, "slab tree factor (height, nodes)", k, cnt)) return SLAB_ESINGULAR;
    }
    return SLAB_OK;
}

// Up pass over all heights for right-hand sides [r0, r0+K) of F (FP64, [k][N]) scaled by fscale,
// then the reduced load f~ into X.
template <typename T>
slab_status tree_up_gather(slab_handle* h, const double* F, double fscale, int r0, int K) {
    SolveArgs<T> p = make_solve_args<T>(h, K);
    const TreeDims& d = h->td;
    SLAB_CK(h, cudaMemsetAsync(h->wFi, 0, (size_t)d.NS * 2 * d.s_pad * h->kcap * h->rsz, h->stream));
    for (int k = 0; k < d.H; ++k) {
        const int cnt = tree_nodes_at(d.s, k);
        if (!cnt) continue;
        dim3 grid(cnt, chunks_at(d.s, k), d.NS);
        SLAB_PROF(h, KC_TREE_UP);
        tree_up_kernel<T><<<grid, TB_THREADS, 0, h->stream>>>(p, k, F, fscale, r0);
        SLAB_CK_LAUNCH(h);
    }
    dim3 g2((unsigned)(((int64_t)d.s_pad * K + 255) / 256), d.NI);
    SLAB_PROF(h, KC_TREE_UP);
    gather_ftilde_kernel<T><<<g2, 256, 0, h->stream>>>(p, F, fscale, r0);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T>
slab_status tree_down_scatter(slab_handle* h, double* U, int accumulate, int r0, int K) {
    SolveArgs<T> p = make_solve_args<T>(h, K);
    const TreeDims& d = h->td;
    for (int k = d.H - 1; k >= 0; --k) {
        const int cnt = tree_nodes_at(d.s, k);
        if (!cnt) continue;
        const int wmax = min(d.s, (1 << (k + 1)) - 1);
        const int dcw = down_chunk(cnt * d.NS, wmax);
        dim3 grid(cnt, (2 * wmax + dcw - 1) / dcw, d.NS);
        SLAB_PROF(h, KC_TREE_DOWN);
        if (h->kind == SLAB_HELMHOLTZ || h->kind == SLAB_CONVECTION)
            tree_down_kernel<T, true><<<grid, TB_THREADS, 0, h->stream>>>(p, k, U, accumulate, r0, (T*)h->wVp,
                                                                          (unsigned*)h->wVtk, dcw);
        else
            tree_down_kernel<T, false><<<grid, TB_THREADS, 0, h->stream>>>(p, k, U, accumulate, r0, (T*)h->wVp,
                                                                           (unsigned*)h->wVtk, dcw);
        SLAB_CK_LAUNCH(h);
    }
    dim3 g2((unsigned)(((int64_t)d.s * K + 255) / 256), d.NI);
    SLAB_PROF(h, KC_TREE_DOWN);
    scatter_utilde_kernel<T><<<g2, 256, 0, h->stream>>>(p, U, accumulate, r0);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T>
slab_status export_ftilde_part(slab_handle* h, double* out, double scale, int r0, int K) {
    SolveArgs<T> p = make_solve_args<T>(h, K);
    const int64_t tot = (int64_t)h->td.NI * h->td.s * K;
    SLAB_PROF(h, KC_OTHER);
    export_x_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(p, out, scale, h->td.NI, r0);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T>
slab_status import_utilde_part(slab_handle* h, const double* in, int r0, int K) {
    SolveArgs<T> p = make_solve_args<T>(h, K);
    const int64_t tot = (int64_t)h->td.NI * h->td.s_pad * K;
    SLAB_PROF(h, KC_OTHER);
    import_x_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(p, in, h->td.NI, r0);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

int tree_kmax() { return KMAX; }

// Scratch elements of the down-pass partial sums (largest height with split nodes) and tickets.
size_t tree_down_ws_elems(int s, int m, int NS) {
    size_t best = 0;
    const int H = tree_height_count(s);
    for (int k = 0; k < H; ++k) {
        const int wmax = min(s, (1 << (k + 1)) - 1);
        const int nch = (2 * wmax + DCW_MIN - 1) / DCW_MIN;
        if (nch <= 1) continue;
        const size_t e = (size_t)NS * tree_nodes_at(s, k) * nch * MAXM * KMAX;
        if (e > best) best = e;
    }
    return best;
}
size_t tree_down_tickets(int s, int NS) { return (size_t)NS * (s / 2 + 1); }

template slab_status tree_factor<float>(slab_handle*);
template slab_status tree_factor<double>(slab_handle*);
template slab_status tree_up_gather<float>(slab_handle*, const double*, double, int, int);
template slab_status tree_up_gather<double>(slab_handle*, const double*, double, int, int);
template slab_status tree_down_scatter<float>(slab_handle*, double*, int, int, int);
template slab_status tree_down_scatter<double>(slab_handle*, double*, int, int, int);
template slab_status export_ftilde_part<float>(slab_handle*, double*, double, int, int);
template slab_status export_ftilde_part<double>(slab_handle*, double*, double, int, int);
template slab_status import_utilde_part<float>(slab_handle*, const double*, int, int);
template slab_status import_utilde_part<double>(slab_handle*, const double*, int, int);
