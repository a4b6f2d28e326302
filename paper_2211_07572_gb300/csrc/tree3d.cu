// Three-dimensional slabs: Stage 1 (Sec. 3.1 in three dimensions), the assembly of T, and the
// parallel phases of Algorithm 4 (eqs. f1-f5 and usol_even).
//
// The slab interior x in [t b + 1, t b + m], y, z in [1, s] is eliminated by cyclic reduction
// along z: a tree row is the sheet z = c of M = m s unknowns (x fastest, then y), the rows form
// the same binary ruler tree as in two dimensions, and a segment [lo, hi] of rows touches the
// contiguous interface range [(lo-1) s, hi s) on each side (interface order: y fastest, then z).
// Each node is a dense M x M elimination; all nodes of one height (over all slabs) form one
// batch of tall matrices (every block row padded to a multiple of 64)
//     [ S ; B_top^T ; B_bot^T ; B_left^T ; B_right^T ; I ]      (M_pad columns)
// eliminated by one batched Cholesky: the rows below S receive (L^{-1} B)^T and the identity
// rows L^{-T}.  The node's condensed top/bottom coupling (R), its top/bottom x interface
// coupling (RI) and its interface x interface Schur product (added into T) follow by batched
// tensor-core products.
#include <algorithm>
#include <vector>

#include "slab_internal.cuh"

struct Tree3Plan {
    int H = 0, M = 0, Mp = 0;
    std::vector<int> cnt, wsp;              // per height: nodes per slab, padded rows of one interface block
    std::vector<int64_t> node_off, zit_off; // per height: first node id, first ZIT element
    int64_t nodes = 0, zit_elems = 0, work_elems = 0, xI_elems = 0;   // xI: per RHS
};

namespace {

constexpr int T3_MAXH = 16;

struct T3Args {
    int n, s, m, M, Mp, NS, sp, b, k, H;
    int cnt[T3_MAXH];
    long long node_off[T3_MAXH];
    const double* AX;
    const double* AY;
    const double* AZ;
    const double* DG;
    __device__ int64_t node(int kk, int t, int i) const { return node_off[kk] + (int64_t)t * cnt[kk] + i; }
    __device__ int64_t coef(int x, int y, int z) const { return ((int64_t)z * (n + 1) + y) * (n + 1) + x; }
};

__device__ inline int t3_right_height(int s, int c, int k) { return tree_right_height(s, c, k); }

// Tall matrix of every node of height A.k: W[node] is rows x Mp, node = t * cnt + i.
template <typename T>
__global__ void t3_build_tall_kernel(T3Args A, int wsp, int rows, T* W, const T* __restrict__ Rtb,
                                     const T* __restrict__ RI) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, m = A.m, M = A.M, Mp = A.Mp, sp = A.sp;
    const int lo = c - (1 << k) + 1, hi = min(s, c + (1 << k) - 1);
    const int w = hi - lo + 1;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = k > 0 ? t3_right_height(s, c, k) : -1;
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    const T* Ra = alpha ? Rtb + A.node(k - 1, t, 2 * i) * 4 * Mp * Mp : nullptr;              // [2Mp][2Mp]
    const T* Rb = beta ? Rtb + A.node(kb, t, ((beta >> kb) - 1) / 2) * 4 * Mp * Mp : nullptr;
    const int x0 = t * A.b + 1;
    T* Wn = W + (int64_t)node * rows * Mp;
    const int ident0 = 3 * Mp + 2 * wsp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)rows * Mp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / Mp), col = (int)(e % Mp);
        T v = T(0);
        if (row < Mp) {                                          // S = D_c + R_alpha[bot,bot] + R_beta[top,top]
            const int r = row, q = col;
            if (r >= M || q >= M) {
                v = r == q ? T(1) : T(0);
            } else {
                const int yr = r / m + 1, xr = r % m, yq = q / m + 1, xq = q % m;
                double d = 0.0;
                if (r == q) d = A.DG[A.coef(x0 + xr, yr, c)];
                else if (yr == yq && (xr - xq == 1 || xq - xr == 1)) d = -A.AX[A.coef(x0 + min(xr, xq), yr, c)];
                else if (xr == xq && (yr - yq == 1 || yq - yr == 1)) d = -A.AY[A.coef(x0 + xr, min(yr, yq), c)];
                v = (T)d;
                if (Ra) v += Ra[(int64_t)(Mp + r) * 2 * Mp + Mp + q];
                if (Rb) v += Rb[(int64_t)r * 2 * Mp + q];
            }
        } else if (row < 3 * Mp) {                               // B_top^T, B_bot^T
            const int bot = row >= 2 * Mp;
            const int j = row - (bot ? 2 * Mp : Mp);             // top / bottom row unknown
            const int q = col;                                   // row-c unknown
            if (j < M && q < M) {
                if (k == 0) {
                    const int zn = bot ? c + 1 : c - 1;
                    if (j == q && zn >= 1 && zn <= s)
                        v = (T)(-A.AZ[A.coef(x0 + q % m, q / m + 1, bot ? c : c - 1)]);
                } else if (!bot && Ra) {
                    v = Ra[(int64_t)j * 2 * Mp + Mp + q];        // alpha's [top, bot]
                } else if (bot && Rb) {
                    v = Rb[(int64_t)(Mp + j) * 2 * Mp + q];      // beta's [bot, top]
                }
            }
        } else if (row < ident0) {                               // B_left^T, B_right^T
            const int side = row >= 3 * Mp + wsp;
            const int loc = row - 3 * Mp - side * wsp;
            const int q = col;
            if (loc < w * s && q < M) {
                const int I = (lo - 1) * s + loc;                // interface index
                const int zI = lo + loc / s, yI = loc % s + 1;
                if (zI == c) {
                    const int yq = q / m + 1, xq = q % m;
                    if (yq == yI) {
                        if (side == 0 && xq == 0 && t >= 1) v = (T)(-A.AX[A.coef(x0 - 1, yq, c)]);
                        if (side == 1 && xq == m - 1 && t < A.NS - 1) v = (T)(-A.AX[A.coef(x0 + m - 1, yq, c)]);
                    }
                } else if (zI < c && alpha) {                    // alpha's bottom row = row c
                    v = RI[((((int64_t)t * A.H + (k - 1)) * 2 + side) * 2 + 1) * Mp * sp + (int64_t)q * sp + I];
                } else if (zI > c && beta) {                     // beta's top row = row c
                    v = RI[((((int64_t)t * A.H + kb) * 2 + side) * 2 + 0) * Mp * sp + (int64_t)q * sp + I];
                }
            }
        } else {
            v = (row - ident0) == col ? T(1) : T(0);
        }
        Wn[e] = v;
    }
}

// Rtb[c] += blockdiag(R_alpha[top,top], R_beta[bot,bot]) after Rtb[c] = -Z_tb^T Z_tb.
template <typename T>
__global__ void t3_add_child_R_kernel(T3Args A, T* Rtb) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int Mp = A.Mp;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = k > 0 ? t3_right_height(A.s, c, k) : -1;
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    if (!alpha && !beta) return;
    T* R = Rtb + A.node(k, t, i) * 4 * Mp * Mp;
    const T* Ra = alpha ? Rtb + A.node(k - 1, t, 2 * i) * 4 * Mp * Mp : nullptr;
    const T* Rb = beta ? Rtb + A.node(kb, t, ((beta >> kb) - 1) / 2) * 4 * Mp * Mp : nullptr;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)Mp * Mp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Mp), q = (int)(e % Mp);
        if (Ra) R[(int64_t)r * 2 * Mp + q] += Ra[(int64_t)r * 2 * Mp + q];
        if (Rb) R[(int64_t)(Mp + r) * 2 * Mp + Mp + q] += Rb[(int64_t)(Mp + r) * 2 * Mp + Mp + q];
    }
}

// RI[t][k][side][top][:, alpha's columns] += RI[t][k-1][side][top]; bottom likewise from beta.
template <typename T>
__global__ void t3_add_child_RI_kernel(T3Args A, T* RI) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, Mp = A.Mp, sp = A.sp;
    const int lo = c - (1 << k) + 1, hi = min(s, c + (1 << k) - 1);
    const int kb = t3_right_height(s, c, k);
    const int nl = (c - lo) * s, nr = (hi - c) * s;              // alpha's and beta's column counts
    for (int side = 0; side < 2; ++side) {
        T* Rt = RI + ((((int64_t)t * A.H + k) * 2 + side) * 2 + 0) * Mp * sp;
        T* Rbt = RI + ((((int64_t)t * A.H + k) * 2 + side) * 2 + 1) * Mp * sp;
        const T* Ca = RI + ((((int64_t)t * A.H + (k - 1)) * 2 + side) * 2 + 0) * Mp * sp;
        const T* Cb = kb >= 0 ? RI + ((((int64_t)t * A.H + kb) * 2 + side) * 2 + 1) * Mp * sp : nullptr;
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)Mp * (nl + nr);
             e += (int64_t)gridDim.x * blockDim.x) {
            const int r = (int)(e / (nl + nr)), j = (int)(e % (nl + nr));
            if (j < nl) {
                const int64_t I = (int64_t)(lo - 1) * s + j;
                Rt[(int64_t)r * sp + I] += Ca[(int64_t)r * sp + I];
            } else if (Cb) {
                const int64_t I = (int64_t)c * s + (j - nl);
                Rbt[(int64_t)r * sp + I] += Cb[(int64_t)r * sp + I];
            }
        }
    }
}

// T_qq = A_qq (the interface plane's stencil, identity padding), T_{q,q+1} = 0 (A_{q,q+1} = 0, b >= 2)
template <typename T>
__global__ void t3_init_T_kernel(T3Args A, T* Tb) {
    const int q = blockIdx.y;
    const int s = A.s, sp = A.sp;
    const int xq = (q + 1) * A.b;
    T* Tq = Tb + (int64_t)q * sp * sp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)sp * sp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(e / sp), J = (int)(e % sp);
        T v = T(0);
        if (I >= s * s || J >= s * s) {
            v = I == J ? T(1) : T(0);
        } else {
            const int yI = I % s + 1, zI = I / s + 1, yJ = J % s + 1, zJ = J / s + 1;
            if (I == J) v = (T)A.DG[A.coef(xq, yI, zI)];
            else if (zI == zJ && (yI - yJ == 1 || yJ - yI == 1)) v = (T)(-A.AY[A.coef(xq, min(yI, yJ), zI)]);
            else if (yI == yJ && (zI - zJ == 1 || zJ - zI == 1)) v = (T)(-A.AZ[A.coef(xq, yI, min(zI, zJ))]);
        }
        Tq[e] = v;
    }
}

// Upper triangle of every diagonal block T_qq from its lower triangle (the interface products
// that add into T_qq are symmetric and computed on the lower tiles only).
template <typename T>
__global__ void t3_mirror_lower_kernel(T* Tb, int sp) {
    T* Tq = Tb + (int64_t)blockIdx.y * sp * sp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)sp * sp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(e / sp), J = (int)(e % sp);
        if (J > I) Tq[e] = Tq[(int64_t)J * sp + I];
    }
}

// ------------------------------------------------------------------ solve kernels
struct T3Vec {
    int kcap, K, r0;
    int64_t N;           // unknowns per right-hand side
};

// g[node][r][j] = fscale f(row c unknown j) + G_alpha[bot] + G_beta[top]
template <typename T>
__global__ void t3_gather_up_kernel(T3Args A, T3Vec V, const double* __restrict__ F, double fscale,
                                    const T* __restrict__ G, T* g) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, m = A.m, M = A.M, Mp = A.Mp;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = k > 0 ? t3_right_height(s, c, k) : -1;
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    const T* Ga = alpha ? G + A.node(k - 1, t, 2 * i) * V.kcap * 2 * Mp : nullptr;
    const T* Gb = beta ? G + A.node(kb, t, ((beta >> kb) - 1) / 2) * V.kcap * 2 * Mp : nullptr;
    T* gn = g + A.node(k, t, i) * V.kcap * Mp;
    const int x0 = t * A.b + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < V.K * Mp; e += gridDim.x * blockDim.x) {
        const int r = e / Mp, j = e % Mp;
        T v = T(0);
        if (j < M) {
            const int y = j / m + 1, x = x0 + j % m;
            v = (T)(fscale * F[(int64_t)(V.r0 + r) * V.N + ((int64_t)(c - 1) * s + (y - 1)) * s + (x - 1)]);
            if (Ga) v += Ga[(int64_t)r * 2 * Mp + Mp + j];
            if (Gb) v += Gb[(int64_t)r * 2 * Mp + j];
        }
        gn[(int64_t)r * Mp + j] = v;
    }
}

// G[node] (after G = -Z_tb^T y) += [G_alpha[top] | G_beta[bot]]
template <typename T>
__global__ void t3_add_child_G_kernel(T3Args A, T3Vec V, T* G) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int Mp = A.Mp;
    const int alpha = k > 0 ? c - (1 << (k - 1)) : 0;
    const int kb = k > 0 ? t3_right_height(A.s, c, k) : -1;
    const int beta = kb >= 0 ? c + (1 << kb) : 0;
    if (!alpha && !beta) return;
    T* Gn = G + A.node(k, t, i) * V.kcap * 2 * Mp;
    const T* Ga = alpha ? G + A.node(k - 1, t, 2 * i) * V.kcap * 2 * Mp : nullptr;
    const T* Gb = beta ? G + A.node(kb, t, ((beta >> kb) - 1) / 2) * V.kcap * 2 * Mp : nullptr;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < V.K * Mp; e += gridDim.x * blockDim.x) {
        const int r = e / Mp, j = e % Mp;
        if (Ga) Gn[(int64_t)r * 2 * Mp + j] += Ga[(int64_t)r * 2 * Mp + j];
        if (Gb) Gn[(int64_t)r * 2 * Mp + Mp + j] += Gb[(int64_t)r * 2 * Mp + Mp + j];
    }
}

// X[q][r][I] = fscale f(interface node I of q) + Fi[q][right][r][I] + Fi[q+1][left][r][I]
template <typename T>
__global__ void t3_gather_ftilde_kernel(T3Args A, T3Vec V, const double* __restrict__ F, double fscale,
                                        const T* __restrict__ Fi, T* X) {
    const int q = blockIdx.y;
    const int s = A.s, sp = A.sp;
    const int xq = (q + 1) * A.b;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)V.K * sp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / sp), I = (int)(e % sp);
        T v = T(0);
        if (I < s * s) {
            const int y = I % s + 1, z = I / s + 1;
            v = (T)(fscale * F[(int64_t)(V.r0 + r) * V.N + ((int64_t)(z - 1) * s + (y - 1)) * s + (xq - 1)]);
            v += Fi[(((int64_t)q * 2 + 1) * V.kcap + r) * sp + I] + Fi[(((int64_t)(q + 1) * 2 + 0) * V.kcap + r) * sp + I];
        }
        X[((int64_t)q * V.kcap + r) * sp + I] = v;
    }
}

// xtb[j][r][0..Mp) = x of the segment's top row, [Mp..2Mp) = x of its bottom row (0 at the boundary)
template <typename T>
__global__ void t3_gather_xtb_kernel(T3Args A, T3Vec V, const T* __restrict__ Xn, T* xtb) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, Mp = A.Mp;
    const int lo = c - (1 << k) + 1, hi = min(s, c + (1 << k) - 1);
    const int top = lo - 1, bot = hi + 1;
    const T* xt = nullptr;
    const T* xb = nullptr;
    if (top >= 1) {
        const int kt = __ffs(top) - 1;
        xt = Xn + A.node(kt, t, ((top >> kt) - 1) / 2) * V.kcap * Mp;
    }
    if (bot <= s) {
        const int kt = __ffs(bot) - 1;
        xb = Xn + A.node(kt, t, ((bot >> kt) - 1) / 2) * V.kcap * Mp;
    }
    T* o = xtb + (int64_t)node * V.kcap * 2 * Mp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < V.K * 2 * Mp; e += gridDim.x * blockDim.x) {
        const int r = e / (2 * Mp), j = e % (2 * Mp);
        T v = T(0);
        if (j < Mp) { if (xt) v = xt[(int64_t)r * Mp + j]; }
        else if (xb) v = xb[(int64_t)r * Mp + (j - Mp)];
        o[(int64_t)r * 2 * Mp + j] = v;
    }
}

// U(row c unknowns) = (or +=) x[node]
template <typename T>
__global__ void t3_scatter_kernel(T3Args A, T3Vec V, const T* __restrict__ Xn, double* U, int accumulate) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, m = A.m, M = A.M, Mp = A.Mp;
    const T* xn = Xn + A.node(k, t, i) * V.kcap * Mp;
    const int x0 = t * A.b + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < V.K * M; e += gridDim.x * blockDim.x) {
        const int r = e / M, j = e % M;
        const int y = j / m + 1, x = x0 + j % m;
        double* up = U + (int64_t)(V.r0 + r) * V.N + ((int64_t)(c - 1) * s + (y - 1)) * s + (x - 1);
        const double v = (double)xn[(int64_t)r * Mp + j];
        if (accumulate) *up += v;
        else *up = v;
    }
}

template <typename T>
__global__ void t3_scatter_utilde_kernel(T3Args A, T3Vec V, const T* __restrict__ X, double* U, int accumulate) {
    const int q = blockIdx.y;
    const int s = A.s, sp = A.sp;
    const int xq = (q + 1) * A.b;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)V.K * s * s;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / (s * s)), I = (int)(e % (s * s));
        const int y = I % s + 1, z = I / s + 1;
        double* up = U + (int64_t)(V.r0 + r) * V.N + ((int64_t)(z - 1) * s + (y - 1)) * s + (xq - 1);
        const double v = (double)X[((int64_t)q * V.kcap + r) * sp + I];
        if (accumulate) *up += v;
        else *up = v;
    }
}

// interface vectors <-> FP64 [k][NI][s^2]
template <typename T>
__global__ void t3_export_kernel(T3Args A, T3Vec V, int NI, const T* __restrict__ X, double* out, double scale) {
    const int64_t si = (int64_t)A.s * A.s;
    const int64_t per = NI * si;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per * V.K;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / per);
        const int64_t rem = e % per;
        const int q = (int)(rem / si);
        const int64_t I = rem % si;
        out[(int64_t)(V.r0 + r) * per + rem] = scale * (double)X[((int64_t)q * V.kcap + r) * A.sp + I];
    }
}
template <typename T>
__global__ void t3_import_kernel(T3Args A, T3Vec V, int NI, const double* __restrict__ in, T* X) {
    const int64_t si = (int64_t)A.s * A.s;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)NI * V.K * A.sp;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(e / ((int64_t)V.K * A.sp));
        const int64_t rem = e % ((int64_t)V.K * A.sp);
        const int r = (int)(rem / A.sp), I = (int)(rem % A.sp);
        X[((int64_t)q * V.kcap + r) * A.sp + I] =
            I < si ? (T)in[(int64_t)(V.r0 + r) * NI * si + (int64_t)q * si + I] : T(0);
    }
}

// xI[j][r][side * wsp + loc] = interface value at column (lo-1) s + loc of the node's segment
// (0 past the segment and for a side without interface)
template <typename T>
__global__ void t3_gather_xI_kernel(T3Args A, T3Vec V, int wsp, const T* __restrict__ X, T* xI) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, sp = A.sp;
    const int lo = c - (1 << k) + 1, hi = min(s, c + (1 << k) - 1);
    const int wl = (hi - lo + 1) * s;
    T* o = xI + (int64_t)node * V.kcap * 2 * wsp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < V.K * 2 * wsp; e += gridDim.x * blockDim.x) {
        const int r = e / (2 * wsp), j = e % (2 * wsp);
        const int side = j >= wsp, loc = j - side * wsp;
        const int q = side ? t : t - 1;
        T v = T(0);
        if (loc < wl && q >= 0 && q < A.NS - 1) v = X[((int64_t)q * V.kcap + r) * sp + (int64_t)(lo - 1) * s + loc];
        o[(int64_t)r * 2 * wsp + j] = v;
    }
}

// Fi[t][side][r][(lo-1) s + loc] += FiN[j][r][side * wsp + loc]   (segments of one height are disjoint)
template <typename T>
__global__ void t3_scatter_Fi_kernel(T3Args A, T3Vec V, int wsp, const T* __restrict__ FiN, T* Fi) {
    const int k = A.k;
    const int node = blockIdx.y;
    const int t = node / A.cnt[k], i = node % A.cnt[k];
    const int c = (2 * i + 1) << k;
    const int s = A.s, sp = A.sp;
    const int lo = c - (1 << k) + 1, hi = min(s, c + (1 << k) - 1);
    const int wl = (hi - lo + 1) * s;
    const T* in = FiN + (int64_t)node * V.kcap * 2 * wsp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < V.K * 2 * wl; e += gridDim.x * blockDim.x) {
        const int r = e / (2 * wl), j = e % (2 * wl);
        const int side = j >= wl, loc = j - side * wl;
        Fi[(((int64_t)t * 2 + side) * V.kcap + r) * sp + (int64_t)(lo - 1) * s + loc] +=
            in[(int64_t)r * 2 * wsp + side * wsp + loc];
    }
}

T3Args make_t3_args(slab_handle* h, int k) {
    const Tree3Plan& P = *h->t3plan;
    T3Args a;
    a.n = h->n; a.s = h->td.s; a.m = h->td.m; a.M = P.M; a.Mp = P.Mp; a.NS = h->td.NS; a.sp = h->td.s_pad;
    a.b = h->b; a.k = k; a.H = P.H;
    for (int i = 0; i < T3_MAXH; ++i) {
        a.cnt[i] = i < P.H ? P.cnt[i] : 0;
        a.node_off[i] = i < P.H ? P.node_off[i] : 0;
    }
    a.AX = h->AX; a.AY = h->AY; a.AZ = h->AZ; a.DG = h->DG;
    return a;
}

inline unsigned grid1(int64_t work) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, 4096)); }

// first node (slab-local index) whose segment is cut by the end of the rows, or cnt if none
inline int first_cut(int s, int k, int cnt) {
    for (int i = 0; i < cnt; ++i)
        if (((2 * i + 1) << k) + (1 << k) - 1 > s) return i;
    return cnt;
}

}  // namespace

// ------------------------------------------------------------------ plan
Tree3Plan* tree3d_plan(int s, int m, int NS) {
    Tree3Plan* P = new Tree3Plan();
    P->H = tree_height_count(s);
    P->M = m * s;
    P->Mp = (P->M + SLAB_TILE - 1) / SLAB_TILE * SLAB_TILE;
    int64_t node = 0, z = 0;
    for (int k = 0; k < P->H; ++k) {
        const int cnt = tree_nodes_at(s, k);
        const int wmax = std::min(s, (1 << (k + 1)) - 1);
        const int wsp = (wmax * s + SLAB_TILE - 1) / SLAB_TILE * SLAB_TILE;
        P->cnt.push_back(cnt);
        P->wsp.push_back(wsp);
        P->node_off.push_back(node);
        P->zit_off.push_back(z);
        node += (int64_t)NS * cnt;
        z += (int64_t)NS * cnt * 2 * wsp * P->Mp;
        const int64_t rows = 4 * (int64_t)P->Mp + 2 * wsp;
        P->work_elems = std::max<int64_t>(P->work_elems, (int64_t)NS * cnt * rows * P->Mp);
        P->xI_elems = std::max<int64_t>(P->xI_elems, (int64_t)NS * cnt * 2 * wsp);
    }
    P->nodes = node;
    P->zit_elems = z;
    return P;
}

void tree3d_plan_free(Tree3Plan* P) { delete P; }
int64_t tree3d_nodes(const Tree3Plan* P) { return P->nodes; }
int tree3d_mpad(const Tree3Plan* P) { return P->Mp; }
int64_t tree3d_zit_elems(const Tree3Plan* P) { return P->zit_elems; }
int64_t tree3d_work_elems(const Tree3Plan* P) { return P->work_elems; }
int64_t tree3d_xI_elems(const Tree3Plan* P) { return P->xI_elems; }

// ------------------------------------------------------------------ factor: Stage 1 and T
template <typename T>
slab_status tree3d_factor(slab_handle* h) {
    const Tree3Plan& P = *h->t3plan;
    const int Mp = P.Mp, NS = h->td.NS, NI = h->td.NI, sp = h->td.s_pad, s = h->td.s;
    const int64_t blk = (int64_t)sp * sp;
    T* Lin = (T*)h->t3Lin;
    T* LT = (T*)h->t3LT;
    T* Ztb = (T*)h->t3Ztb;
    T* ZtbT = (T*)h->t3ZtbT;
    T* ZIT = (T*)h->t3ZIT;
    T* ZI = (T*)h->t3ZI;
    T* Rtb = (T*)h->t3Rtb;
    T* RI = (T*)h->t3RI;
    T* W = (T*)h->t3W;
    T* Tb = (T*)h->Tb;
    T* To = (T*)h->To;
    slab_status st;
    {
        T3Args a = make_t3_args(h, 0);
        SLAB_PROF(h, KC_ASSEMBLE);
        t3_init_T_kernel<T><<<dim3(grid1(blk), NI), 256, 0, h->stream>>>(a, Tb);
        SLAB_CK_LAUNCH(h);
        if (NI > 1) SLAB_CK(h, cudaMemsetAsync(To, 0, (size_t)(NI - 1) * blk * sizeof(T), h->stream));
    }
    for (int k = 0; k < P.H; ++k) {
        const int cnt = P.cnt[k];
        if (!cnt) continue;
        const int B = NS * cnt;
        const int wsp = P.wsp[k];
        const int rows = 4 * Mp + 2 * wsp;
        const int ident0 = 3 * Mp + 2 * wsp;
        const int64_t wstride = (int64_t)rows * Mp;
        T3Args a = make_t3_args(h, k);
        const int64_t n0 = P.node_off[k];
        {
            SLAB_PROF(h, KC_TREE_FACTOR);
            t3_build_tall_kernel<T><<<dim3(grid1(wstride) < 64 ? grid1(wstride) : 64, B), 256, 0, h->stream>>>(
                a, wsp, rows, W, Rtb, RI);
            SLAB_CK_LAUNCH(h);
        }
        if ((st = dense_tall_cholesky<T>(h, W, Mp, ident0, B, wstride))) return st;
        if (slab_debug() && slab_debug_status(h, "3-D slab tree factor (height, nodes)", k, B)) return SLAB_ESINGULAR;
        // factors of the solve: L^{-T}, L^{-1}, (Z_tb)^T, Z_tb, (Z_I)^T, Z_I
        const int64_t mm = (int64_t)Mp * Mp;
        if ((st = dense_copy<T>(h, W + (int64_t)ident0 * Mp, wstride, LT + n0 * mm, mm, mm, B))) return st;
        if ((st = dense_transpose<T>(h, LT + n0 * mm, Mp, mm, Lin + n0 * mm, Mp, mm, Mp, Mp, B))) return st;
        if ((st = dense_copy<T>(h, W + (int64_t)Mp * Mp, wstride, ZtbT + n0 * 2 * mm, 2 * mm, 2 * mm, B))) return st;
        if ((st = dense_transpose<T>(h, ZtbT + n0 * 2 * mm, Mp, 2 * mm, Ztb + n0 * 2 * mm, 2 * Mp, 2 * mm, 2 * Mp, Mp,
                                     B)))
            return st;
        T* zit = ZIT + P.zit_off[k];
        const int64_t zs = (int64_t)2 * wsp * Mp;
        if ((st = dense_copy<T>(h, W + (int64_t)3 * Mp * Mp, wstride, zit, zs, zs, B))) return st;
        if ((st = dense_transpose<T>(h, zit, Mp, zs, ZI + P.zit_off[k], 2 * wsp, zs, 2 * wsp, Mp, B))) return st;
        // condensed top / bottom rows for the parent: Rtb = -Z_tb^T Z_tb (+ children), RI = -Z_tb^T Z_I (+ children)
        const int64_t rs = 4 * mm;
        if ((st = dense_gemm<T>(h, KC_SYRK, 2 * Mp, 2 * Mp, Mp, T(-1), ZtbT + n0 * 2 * mm, Mp, 2 * mm,
                                ZtbT + n0 * 2 * mm, Mp, 2 * mm, T(0), Rtb + n0 * rs, 2 * Mp, rs, 0, 0, B)))
            return st;
        {
            SLAB_PROF(h, KC_OTHER);
            t3_add_child_R_kernel<T><<<dim3(grid1(mm) < 64 ? grid1(mm) : 64, B), 256, 0, h->stream>>>(a, Rtb);
            SLAB_CK_LAUNCH(h);
        }
        const int cut = first_cut(s, k, cnt);
        for (int t = 0; t < NS; ++t) {
            for (int side = 0; side < 2; ++side) {
                T* RIo = RI + (((int64_t)t * P.H + k) * 2 + side) * 2 * Mp * sp;      // [tb][Mp][sp] = 2Mp rows
                // full nodes as one strided batch, the cut node alone
                for (int part = 0; part < 2; ++part) {
                    const int i0 = part == 0 ? 0 : cut;
                    const int nb = part == 0 ? cut : cnt - cut;
                    if (nb <= 0) continue;
                    const int c = (2 * i0 + 1) << k;
                    const int lo = c - (1 << k) + 1, hi = std::min(s, c + (1 << k) - 1);
                    const int wl = (hi - lo + 1) * s;
                    const int64_t nd = n0 + (int64_t)t * cnt + i0;
                    const T* zI = zit + ((int64_t)(t * cnt + i0) * 2 + side) * wsp * Mp;
                    const int64_t colstep = (int64_t)(2 << k) * s;
                    if ((st = dense_gemm<T>(h, KC_SYRK, 2 * Mp, wl, Mp, T(-1), ZtbT + nd * 2 * mm, Mp, 2 * mm, zI, Mp, zs,
                                            T(0), RIo + (int64_t)(lo - 1) * s, sp, colstep, 0, 0, nb)))
                        return st;
                }
            }
        }
        if (k > 0) {
            SLAB_PROF(h, KC_OTHER);
            t3_add_child_RI_kernel<T><<<dim3(256, B), 256, 0, h->stream>>>(a, RI);
            SLAB_CK_LAUNCH(h);
        }
        // T += -Z_I^T Z_I of every node: slab t's right side into T_tt, left side into T_{t-1,t-1},
        // left x right into T_{t-1,t}
        for (int t = 0; t < NS; ++t) {
            for (int pair = 0; pair < 3; ++pair) {
                const int sa = pair == 0 ? 1 : 0, sb = pair == 2 ? 1 : (pair == 0 ? 1 : 0);
                T* Tq;
                if (pair == 0) { if (t >= NI) continue; Tq = Tb + (int64_t)t * blk; }
                else if (pair == 1) { if (t < 1) continue; Tq = Tb + (int64_t)(t - 1) * blk; }
                else { if (t < 1 || t >= NI) continue; Tq = To + (int64_t)(t - 1) * blk; }
                for (int part = 0; part < 2; ++part) {
                    const int i0 = part == 0 ? 0 : cut;
                    const int nb = part == 0 ? cut : cnt - cut;
                    if (nb <= 0) continue;
                    const int c = (2 * i0 + 1) << k;
                    const int lo = c - (1 << k) + 1, hi = std::min(s, c + (1 << k) - 1);
                    const int wl = (hi - lo + 1) * s;
                    const T* za = zit + ((int64_t)(t * cnt + i0) * 2 + sa) * wsp * Mp;
                    const T* zb = zit + ((int64_t)(t * cnt + i0) * 2 + sb) * wsp * Mp;
                    const int64_t off = (int64_t)(lo - 1) * s;
                    const int64_t step = (int64_t)(2 << k) * s;
                    // pairs 0 and 1 add a symmetric product into a diagonal block: lower tiles only
                    if ((st = dense_gemm<T>(h, KC_ASSEMBLE, wl, wl, Mp, T(-1), za, Mp, zs, zb, Mp, zs, T(1),
                                            Tq + off * sp + off, sp, step * sp + step, 0, pair < 2, nb)))
                        return st;
                }
            }
        }
    }
    {
        SLAB_PROF(h, KC_ASSEMBLE);
        t3_mirror_lower_kernel<T><<<dim3(grid1(blk) < 256 ? grid1(blk) : 256, NI), 256, 0, h->stream>>>(Tb, sp);
        SLAB_CK_LAUNCH(h);
    }
    return SLAB_OK;
}

// ------------------------------------------------------------------ solve phases
// Up pass (eqs. f1-f5) for right-hand sides [r0, r0+K) of F scaled by fscale; the reduced load into wX.
template <typename T>
slab_status tree3d_up_gather(slab_handle* h, const double* F, double fscale, int r0, int K) {
    const Tree3Plan& P = *h->t3plan;
    const int Mp = P.Mp, NS = h->td.NS, NI = h->td.NI, sp = h->td.s_pad, s = h->td.s, kc = h->kcap;
    const int64_t mm = (int64_t)Mp * Mp;
    T* y = (T*)h->t3y;
    T* G = (T*)h->t3G;
    T* g = (T*)h->t3x;              // the x buffer holds g during the up pass
    T* Fi = (T*)h->t3Fi;
    T3Vec V{kc, K, r0, (int64_t)s * s * s};
    slab_status st;
    SLAB_CK(h, cudaMemsetAsync(Fi, 0, (size_t)NS * 2 * kc * sp * sizeof(T), h->stream));
    for (int k = 0; k < P.H; ++k) {
        const int cnt = P.cnt[k];
        if (!cnt) continue;
        const int B = NS * cnt;
        const int64_t n0 = P.node_off[k];
        T3Args a = make_t3_args(h, k);
        {
            SLAB_PROF(h, KC_TREE_UP);
            t3_gather_up_kernel<T><<<dim3(grid1((int64_t)K * Mp) < 32 ? grid1((int64_t)K * Mp) : 32, B), 256, 0,
                                     h->stream>>>(a, V, F, fscale, G, g);
            SLAB_CK_LAUNCH(h);
        }
        // y = L^{-1} g  (L^{-1} lower triangular: each row tile reads only its nonzero part)
        if ((st = dense_gemm<T>(h, KC_TREE_UP, Mp, K, Mp, T(1), (T*)h->t3Lin + n0 * mm, Mp, mm, g + n0 * kc * Mp, Mp,
                                (int64_t)kc * Mp, T(0), y + n0 * kc * Mp, Mp, (int64_t)kc * Mp, 1, 0, B, 1)))
            return st;
        // G = -Z_tb^T y (+ children's outer loads)
        if ((st = dense_gemm<T>(h, KC_TREE_UP, 2 * Mp, K, Mp, T(-1), (T*)h->t3ZtbT + n0 * 2 * mm, Mp, 2 * mm,
                                y + n0 * kc * Mp, Mp, (int64_t)kc * Mp, T(0), G + n0 * kc * 2 * Mp, 2 * Mp,
                                (int64_t)kc * 2 * Mp, 1, 0, B)))
            return st;
        {
            SLAB_PROF(h, KC_TREE_UP);
            t3_add_child_G_kernel<T><<<dim3(grid1((int64_t)K * Mp) < 32 ? grid1((int64_t)K * Mp) : 32, B), 256, 0,
                                       h->stream>>>(a, V, G);
            SLAB_CK_LAUNCH(h);
        }
        // Fi[t][side] -= Z_I^T y over the segment's interface columns (per node, then scattered)
        const int wsp = P.wsp[k];
        const int64_t zs = (int64_t)2 * wsp * Mp;
        T* FiN = (T*)h->t3xI;
        if ((st = dense_gemm<T>(h, KC_TREE_UP, 2 * wsp, K, Mp, T(-1), (const T*)h->t3ZIT + P.zit_off[k], Mp, zs,
                                y + n0 * kc * Mp, Mp, (int64_t)kc * Mp, T(0), FiN, 2 * wsp, (int64_t)kc * 2 * wsp, 1, 0,
                                B)))
            return st;
        {
            SLAB_PROF(h, KC_TREE_UP);
            t3_scatter_Fi_kernel<T><<<dim3(grid1((int64_t)K * 2 * wsp) < 64 ? grid1((int64_t)K * 2 * wsp) : 64, B),
                                      256, 0, h->stream>>>(a, V, wsp, FiN, Fi);
            SLAB_CK_LAUNCH(h);
        }
    }
    T3Args a = make_t3_args(h, 0);
    SLAB_PROF(h, KC_TREE_UP);
    t3_gather_ftilde_kernel<T><<<dim3(grid1((int64_t)K * sp), NI), 256, 0, h->stream>>>(a, V, F, fscale, Fi,
                                                                                        (T*)h->wX);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

// Down pass (eq. usol_even) from the interface values in wX; U = (or +=) the solution.
template <typename T>
slab_status tree3d_down_scatter(slab_handle* h, double* U, int accumulate, int r0, int K) {
    const Tree3Plan& P = *h->t3plan;
    const int Mp = P.Mp, NS = h->td.NS, NI = h->td.NI, s = h->td.s, kc = h->kcap;
    const int64_t mm = (int64_t)Mp * Mp;
    T* y = (T*)h->t3y;
    T* X = (T*)h->t3x;
    T* xtb = (T*)h->t3G;            // the G buffer holds the outer x values during the down pass
    const T* Xi = (const T*)h->wX;
    T3Vec V{kc, K, r0, (int64_t)s * s * s};
    slab_status st;
    for (int k = P.H - 1; k >= 0; --k) {
        const int cnt = P.cnt[k];
        if (!cnt) continue;
        const int B = NS * cnt;
        const int64_t n0 = P.node_off[k];
        T3Args a = make_t3_args(h, k);
        {
            SLAB_PROF(h, KC_TREE_DOWN);
            t3_gather_xtb_kernel<T><<<dim3(grid1((int64_t)K * 2 * Mp) < 32 ? grid1((int64_t)K * 2 * Mp) : 32, B), 256,
                                      0, h->stream>>>(a, V, X, xtb);
            SLAB_CK_LAUNCH(h);
        }
        // V = y - Z_tb x_tb - Z_I u_I  (in place in y), x = L^{-T} V
        if ((st = dense_gemm<T>(h, KC_TREE_DOWN, Mp, K, 2 * Mp, T(-1), (T*)h->t3Ztb + n0 * 2 * mm, 2 * Mp, 2 * mm, xtb,
                                2 * Mp, (int64_t)kc * 2 * Mp, T(1), y + n0 * kc * Mp, Mp, (int64_t)kc * Mp, 1, 0, B)))
            return st;
        const int wsp = P.wsp[k];
        T* xI = (T*)h->t3xI;
        {
            SLAB_PROF(h, KC_TREE_DOWN);
            t3_gather_xI_kernel<T><<<dim3(grid1((int64_t)K * 2 * wsp) < 64 ? grid1((int64_t)K * 2 * wsp) : 64, B), 256,
                                     0, h->stream>>>(a, V, wsp, Xi, xI);
            SLAB_CK_LAUNCH(h);
        }
        if ((st = dense_gemm<T>(h, KC_TREE_DOWN, Mp, K, 2 * wsp, T(-1), (const T*)h->t3ZI + P.zit_off[k], 2 * wsp,
                                (int64_t)2 * wsp * Mp, xI, 2 * wsp, (int64_t)kc * 2 * wsp, T(1), y + n0 * kc * Mp, Mp,
                                (int64_t)kc * Mp, 1, 0, B)))
            return st;
        if ((st = dense_gemm<T>(h, KC_TREE_DOWN, Mp, K, Mp, T(1), (T*)h->t3LT + n0 * mm, Mp, mm, y + n0 * kc * Mp, Mp,
                                (int64_t)kc * Mp, T(0), X + n0 * kc * Mp, Mp, (int64_t)kc * Mp, 1, 0, B, 2)))
            return st;
        {
            SLAB_PROF(h, KC_TREE_DOWN);
            t3_scatter_kernel<T><<<dim3(grid1((int64_t)K * P.M) < 32 ? grid1((int64_t)K * P.M) : 32, B), 256, 0,
                                   h->stream>>>(a, V, X, U, accumulate);
            SLAB_CK_LAUNCH(h);
        }
    }
    T3Args a = make_t3_args(h, 0);
    SLAB_PROF(h, KC_TREE_DOWN);
    t3_scatter_utilde_kernel<T><<<dim3(grid1((int64_t)K * s * s), NI), 256, 0, h->stream>>>(a, V, Xi, U, accumulate);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T>
slab_status tree3d_export(slab_handle* h, double* out, double scale, int r0, int K) {
    T3Args a = make_t3_args(h, 0);
    T3Vec V{h->kcap, K, r0, 0};
    SLAB_PROF(h, KC_OTHER);
    t3_export_kernel<T><<<grid1((int64_t)h->td.NI * h->td.s * h->td.s * K), 256, 0, h->stream>>>(
        a, V, h->td.NI, (const T*)h->wX, out, scale);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template <typename T>
slab_status tree3d_import(slab_handle* h, const double* in, int r0, int K) {
    T3Args a = make_t3_args(h, 0);
    T3Vec V{h->kcap, K, r0, 0};
    SLAB_PROF(h, KC_OTHER);
    t3_import_kernel<T><<<grid1((int64_t)h->td.NI * h->td.s_pad * K), 256, 0, h->stream>>>(a, V, h->td.NI, in,
                                                                                         (T*)h->wX);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template slab_status tree3d_factor<float>(slab_handle*);
template slab_status tree3d_factor<double>(slab_handle*);
template slab_status tree3d_up_gather<float>(slab_handle*, const double*, double, int, int);
template slab_status tree3d_up_gather<double>(slab_handle*, const double*, double, int, int);
template slab_status tree3d_down_scatter<float>(slab_handle*, double*, int, int, int);
template slab_status tree3d_down_scatter<double>(slab_handle*, double*, int, int, int);
template slab_status tree3d_export<float>(slab_handle*, double*, double, int, int);
template slab_status tree3d_export<double>(slab_handle*, double*, double, int, int);
template slab_status tree3d_import<float>(slab_handle*, const double*, int, int);
template slab_status tree3d_import<double>(slab_handle*, const double*, int, int);
