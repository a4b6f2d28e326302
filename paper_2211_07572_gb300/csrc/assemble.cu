// Assembly of the reduced matrix T (Sec. 3.1, eqs. T11-T35), fused with the
// interface x interface part of every slab Schur complement.
//
// For slab t the condensed matrix on its interface nodes is
//   M_t[p,p'] = - sum_{heights k} [p, p' in the same height-k segment] Z_{t,k}[:,p] . Z_{t,k}[:,p'],
// where Z_{t,k} (m x s per slab side) holds the Z = L^{-1} B columns of the
// height-k separators (zero for rows no height-k node owns); for the indefinite kind the
// product is B_{t,k}[:,p] . W_{t,k}[:,p'] with W = S^{-1} B, and for the nonsymmetric kind
// C^T_{t,k}[:,p] . W_{t,k}[:,p'] (C the couplings of the interface rows into the separators).  Then
//   T_qq      = A_qq + M_q[R,R] + M_{q+1}[L,L],      T_{q,q+1} = M_{q+1}[L,R]
// (A_{q,q+1} = 0 for b >= 2), and for the nonsymmetric kind also T_{q+1,q} = M_{q+1}[R,L].  Each 64 x 64 output tile is written once; with
// 64-aligned tiles, heights k >= 5 need no mask (a tile lies inside one
// segment), heights k < 5 only touch diagonal tiles.  HBM traffic is the T
// write (the Z operands are re-read from L2).
#include "slab_internal.cuh"

namespace {

template <typename T>
struct AsmArgs {
    int s, s_pad, m, H, NS, NI, b, n;
    const double* AY;
    const double* AYT;   // nonsymmetric kind: -h^2 A[(x,y+1),(x,y)] (else AY)
    const double* DG;
    const T* ZI;       // left factors: Z (SPD kinds) or B (indefinite kind)
    const T* ZR;       // right factors: Z (SPD kinds) or W = S^{-1} B (indefinite kind)
    T* Tb;
    T* To;
    T* Tl;             // nonsymmetric kind: T_{q+1,q} (else null)
    __device__ const T* zi(int t, int k, int side) const {
        return ZI + (((int64_t)t * H + k) * 2 + side) * m * s_pad;
    }
    __device__ const T* zr(int t, int k, int side) const {
        return ZR + (((int64_t)t * H + k) * 2 + side) * m * s_pad;
    }
};

template <typename T>
__device__ void add_contribution(const AsmArgs<T>& A, int t, int sa, int sb, int u, int v, T acc[4][4],
                                 T* sA, T* sB) {
    const int tid = threadIdx.x;
    const int ty = tid / 16, tx = tid % 16;
    const int m = A.m;
    for (int k = 0; k < A.H; ++k) {
        bool masked;
        if (k >= 5) {
            if ((u >> (k - 5)) != (v >> (k - 5))) continue;
            masked = false;
        } else {
            if (u != v) continue;
            masked = true;
        }
        const T* za = A.zi(t, k, sa) + (int64_t)u * SLAB_TILE;
        const T* zb = A.zr(t, k, sb) + (int64_t)v * SLAB_TILE;
        __syncthreads();
        for (int idx = tid; idx < m * SLAB_TILE; idx += blockDim.x) {
            const int i = idx / SLAB_TILE, j = idx % SLAB_TILE;
            sA[i * SLAB_TILE + j] = za[(int64_t)i * A.s_pad + j];
            sB[i * SLAB_TILE + j] = zb[(int64_t)i * A.s_pad + j];
        }
        __syncthreads();
        T p[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) p[a][b2] = T(0);
        for (int i = 0; i < m; ++i) {
            T av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sA[i * SLAB_TILE + ty + 16 * a];
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) bv[b2] = sB[i * SLAB_TILE + tx + 16 * b2];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b2 = 0; b2 < 4; ++b2) p[a][b2] += av[a] * bv[b2];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b2 = 0; b2 < 4; ++b2) {
                const int r = ty + 16 * a, r2 = tx + 16 * b2;
                if (!masked || (r >> (k + 1)) == (r2 >> (k + 1))) acc[a][b2] -= p[a][b2];
            }
    }
}

// grid = (tile col v, tile row u, block z): z < NI -> T_qq (q = z), z < 2 NI - 1 -> T_{q,q+1}
// (q = z - NI), else T_{q+1,q} (q = z - 2 NI + 1, nonsymmetric kind)
template <typename T>
__global__ void __launch_bounds__(256) assemble_T_kernel(AsmArgs<T> A) {
    __shared__ T sA[SLAB_MAXM * SLAB_TILE];
    __shared__ T sB[SLAB_MAXM * SLAB_TILE];
    const int v = blockIdx.x, u = blockIdx.y, z = blockIdx.z;
    const bool diag = z < A.NI;
    const bool lower = z >= 2 * A.NI - 1;
    const int q = diag ? z : (lower ? z - (2 * A.NI - 1) : z - A.NI);
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = T(0);
    if (diag) {
        add_contribution<T>(A, q, 1, 1, u, v, acc, sA, sB);        // slab q, right side
        add_contribution<T>(A, q + 1, 0, 0, u, v, acc, sA, sB);    // slab q+1, left side
    } else if (!lower) {
        add_contribution<T>(A, q + 1, 0, 1, u, v, acc, sA, sB);    // slab q+1, left x right
    } else {
        add_contribution<T>(A, q + 1, 1, 0, u, v, acc, sA, sB);    // slab q+1, right x left
    }
    T* out = (diag ? A.Tb : (lower ? A.Tl : A.To)) + (int64_t)q * A.s_pad * A.s_pad;
    const int xq = (q + 1) * A.b;
    const int np1 = A.n + 1;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) {
            const int r = u * SLAB_TILE + ty + 16 * a;
            const int r2 = v * SLAB_TILE + tx + 16 * b2;
            T val = acc[a][b2];
            if (diag) {
                if (r == r2) val += r < A.s ? (T)A.DG[(int64_t)(r + 1) * np1 + xq] : T(1);
                else if (r2 == r + 1 && r2 < A.s)
                    val -= (T)A.AY[(int64_t)(r + 1) * np1 + xq];           // A[(xq,r+1),(xq,r+2)]
                else if (r == r2 + 1 && r < A.s)
                    val -= (T)A.AYT[(int64_t)(r2 + 1) * np1 + xq];         // A[(xq,r+1),(xq,r)]
            }
            out[(int64_t)r * A.s_pad + r2] = val;
        }
}

}  // namespace

template <typename T>
slab_status assemble_T(slab_handle* h) {
    AsmArgs<T> a;
    const TreeDims& d = h->td;
    a.s = d.s; a.s_pad = d.s_pad; a.m = d.m; a.H = d.H; a.NS = d.NS; a.NI = d.NI; a.b = h->b; a.n = h->n;
    a.AY = h->AY; a.DG = h->DG; a.ZI = (const T*)h->tZI; a.Tb = (T*)h->Tb; a.To = (T*)h->To;
    a.ZR = (h->kind == SLAB_HELMHOLTZ || h->kind == SLAB_CONVECTION) ? (const T*)h->tWI : (const T*)h->tZI;
    const bool ns = h->kind == SLAB_CONVECTION;
    a.AYT = ns ? h->AYT : h->AY;
    a.Tl = ns ? (T*)h->Tl : nullptr;
    const int nt = h->nt;
    dim3 grid(nt, nt, d.NI + (d.NI - 1) * (ns ? 2 : 1));
    SLAB_PROF(h, KC_ASSEMBLE);
    assemble_T_kernel<T><<<grid, 256, 0, h->stream>>>(a);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

template slab_status assemble_T<float>(slab_handle*);
template slab_status assemble_T<double>(slab_handle*);
