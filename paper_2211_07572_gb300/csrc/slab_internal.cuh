// Internal declarations of the slab factor+solve library (CUDA, sm_103a).
//
// Internal operator scaling: all factor data describe Ahat = h^2 A, so the
// stencil entries are O(kappa) and the right-hand sides are h^2 f.
//
// Geometry (2-D).  Rows y = 1..s (s = n-1).  Slab t (0-based, t < NS = n/b)
// holds the interior columns x = t b + 1 .. t b + m (m = b-1); interface q
// (0-based, q < NI = NS-1) is the column x = (q+1) b, the right interface of
// slab q and the left interface of slab q+1.
//
// Slab-interior elimination order: the rows of a slab are eliminated along a
// binary "ruler" tree -- row c has height k = ctz(c); node c owns the segment
// [c - 2^k + 1, min(s, c + 2^k - 1)] and is eliminated after its children
// (cyclic reduction along y).  Eliminating node c condenses its segment onto
// the row above the segment ("top"), the row below ("bot") and the interface
// nodes of the segment's rows on both slab sides.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "slab.h"

#define SLAB_TILE 64
#define SLAB_MAXM 32          // largest slab interior width handled by the 2-D tree kernels
#define SLAB_SPLITK 8         // K splits of the skinny solve products

// Bytes of the split-K partial-sum buffer of a handle whose interfaces have s_pad nodes:
// [s_pad/64][SLAB_SPLITK][64][64] FP64 tiles (FP32 products use it as a flat float array).
inline size_t splitk_part_bytes(int s_pad) {
    return (size_t)(s_pad / SLAB_TILE) * SLAB_SPLITK * SLAB_TILE * SLAB_TILE * 8;
}

// Device-side status word bits (set by kernels, read by the host after a phase).
#define SLAB_DEV_NOTSPD 1u    // a Cholesky pivot was <= 0 or not finite
#define SLAB_DEV_TIMEOUT 2u   // a bounded device-side wait gave up (tensor-core pipeline)

// Diagnostics: with the environment variable SLAB_DEBUG set, the factor synchronises after each
// phase step and reports on stderr where a pivot failure first appeared.
bool slab_debug();
unsigned slab_debug_status(slab_handle* h, const char* where, int a, int b);

struct TreeDims {
    int s;        // rows per slab, n - 1 (= interface size in 2-D)
    int si;       // interface unknowns (n-1)^(d-1)
    int64_t N;    // unknowns (n-1)^d
    int s_pad;    // si rounded up to SLAB_TILE
    int m;        // slab interior width
    int H;        // tree heights 0..H-1
    int NS, NI;   // slabs, interfaces
    int b, n;
};

// Bump allocator over one device region; handles created in it never free their buffers (the
// region's owner frees it).  With base == nullptr it only adds up the bytes (a sizing pass).
struct SlabArena {
    char* base;
    size_t off, cap;
};

struct slab_handle {
    int dim, n, b, kind;
    SlabArena* arena;         // non-null: every device buffer comes from this arena
    double omega;
    int prec;                 // slab_precision of Stage 1 (slab trees, T assembly, tree solves)
    size_t rsz;               // bytes of the Stage-1 scalar
    int prec2;                // slab_precision of Stage 2 (interface elimination and sweep)
    int tf32;                 // SLAB_PREC_TF32 requested: single-pass TF32 products in the factor
    int tf32_now;             // set while the factor runs
    int fp64tc;               // SLAB_PREC_FP64_TC interface: FP64 products of Stage 2 on the tensor cores
    int fp64tc_now;           // set while the interface elimination runs
    void* ozw;                // work area of those products
    void* w16;                // FP32 factor: operand splits of the FP16 three-product path (factor only)
    size_t w16_bytes;
    void* pnl;                // panel inverses of the tall Cholesky (factor only)
    size_t pnl_bytes;
    size_t rsz2;              // bytes of the Stage-2 scalar
    void *Tb1, *To1;          // mixed mode: T assembled in the Stage-1 scalar (factor only)
    void *wX2, *wZ2;          // mixed mode: interface vectors in the Stage-2 scalar
    TreeDims td;
    int nt;                   // tiles per interface block (s_pad / 64)
    cudaStream_t stream;
    int own_stream;           // the stream was created for this handle (batched factor)
    double rtol;
    int max_refine;
    int krylov;               // 0: plain refinement; m > 0: restarted GMRES(m) refinement
    double* kV;               // Krylov basis [m+1][k][N] (FP64)
    double* kZ;               // preconditioned directions [m][k][N] (FP64)
    double* kS;               // small device arrays: H columns, coefficients, dot partials
    int kcapk;                // k the Krylov arrays were sized for

    // coefficient arrays over the (n+1)^2 nodes, h^2-scaled, FP64
    double* AX;               // AX[y][x]: face (x,y)-(x+1,y)
    double* AY;               // AY[y][x]: face (x,y)-(x,y+1)
    double* DG;               // DG[y][x]: diagonal of Ahat at (x,y)
    double* kappa;            // copy of the node coefficient (DIFFUSION, CONVECTION), for the gradient
    double* AXT;              // CONVECTION: AXT[y][x] = -h^2 A[(x+1,y),(x,y)] (AX: -h^2 A[(x,y),(x+1,y)])
    double* AYT;              // CONVECTION: AYT[y][x] = -h^2 A[(x,y+1),(x,y)] (AY: -h^2 A[(x,y),(x,y+1)])
    int transposed;           // set while a solve with A^T runs (CONVECTION adjoint)
    int pivot_local;          // Gauss-Jordan sweep: pivot rows from the diagonal 64-row block only
    const double* beta;       // CONVECTION: the caller's velocity field, set during slab_factor only
    double* AZ;               // 3-D: AZ[z][y][x]: face (x,y,z)-(x,y,z+1)

    // 3-D Stage 1 (tree3d.cu): per-node dense factors, node ids height-major (see Tree3Plan)
    struct Tree3Plan* t3plan;
    void *t3Lin, *t3LT;       // [node][Mp][Mp]  L^{-1}, L^{-T}
    void *t3Ztb, *t3ZtbT;     // [node][Mp][2Mp] Z_tb = L^{-1} B_tb, and its transpose
    void *t3ZIT, *t3ZI;       // per height [node][2 wsp][Mp] (Z_I)^T and [node][Mp][2 wsp] Z_I
    void *t3Rtb, *t3RI, *t3W; // factor only: condensed R [node][2Mp][2Mp], RI [t][k][side][tb][Mp][s_pad], work
    void *t3y, *t3G, *t3x, *t3Fi, *t3xI;   // solve workspace

    // Stage-1 factors (scalar = float or double)
    void* tLinv;              // [NS][s+1][m*m]   inverse Cholesky factor of each separator row
    void* tZtb;               // [NS][s+1][m*2m]  Z = Linv B for the top/bot rows
    void* tRtb;               // [NS][s+1][2m*2m] condensed top/bot x top/bot block
    void* tZI;                // [NS][H][2][m][s_pad]  Z for interface nodes, per height
    void* tRI;                // [NS][H][2][2][m][s_pad] condensed top/bot x interface rows
    void* tWtb;               // Helmholtz only: [NS][s+1][m*2m] W = S^{-1} B (top/bot columns)
    void* tWI;                // Helmholtz only: [NS][H][2][m][s_pad] W for the interface columns
    void* ToT;                // Helmholtz only: [NI-1][s_pad][s_pad] T_{q+1,q} (row-major)
    // CONVECTION only: the elimination of A^T from the same tree (see tree.cu), and Stage 2's
    // T_{q+1,q} plus the transposed factors of the A^T sweep
    void *tLinvT, *tZtbT, *tWtbT, *tZIT, *tWIT, *tRIc;
    void* Tl;                 // [NI-1][s_pad][s_pad] T_{q+1,q} as assembled (Stage-2 scalar)
    void* Tl1;                // mixed mode: T_{q+1,q} in the Stage-1 scalar (factor only)
    void *SinvT, *WT, *TlT;   // S_j^{-T}, W_j^T, T_{j+1,j}^T (Stage-2 scalar)
    int stage2;               // 0: sequential sweep (Algorithm 1), 1: odd-even elimination order
    void *crD, *crE, *crW, *crLT, *crPt, *crP, *crQt, *crQ;   // odd-even order storage

    // Stage-2 data
    void* Tb;                 // [NI][s_pad][s_pad]  T_qq (kept as assembled)
    void* To;                 // [NI-1][s_pad][s_pad] T_{q,q+1}
    void* Fct;                // [NI][3][s_pad][s_pad]: S_j (then L_j), L_j^{-T}, Y_j^T
    void* Linv;               // [NI][s_pad][s_pad] L_j^{-1}, S_j = L_j L_j^T
    void* Y;                  // [NI-1][s_pad][s_pad] Y_j = L_j^{-1} T_{j,j+1}

    unsigned int* dstatus;    // device status word
    void* dscratch;           // 256 bytes of device scratch
    void* gjw;                // indefinite kind: Stage-2 Gauss-Jordan work area (gj_work_bytes)

    // solve workspace, sized for kcap right-hand sides
    int kcap;
    void* wYv;                // [NS][s+1][m][k]     y of each separator (up pass)
    void* wGtb;               // [NS][s+1][2][m][k]  condensed top/bot load
    void* wXs;                // [NS][s+1][m][k]     interior solution per row
    void* wFi;                // [NS][2][s_pad][k]   interface load contributions
    void* wX;                 // [NI][k][s_pad]  interface vectors, right-hand-side major
    void* wZ;                 // [NI][k][s_pad]
    void* wVp;                // down-pass partial sums of split nodes
    void* wVtk;               // down-pass tickets (self-resetting)
    void* wPart;              // [s_pad/64][SLAB_SPLITK][64][64] skinny-product partial tiles
    unsigned* wTickets;       // [s_pad/64] self-resetting tile counters
    double* wR;               // [rcap][N] FP64 residual
    double* wNrm;             // [2 rcap] FP64 norms
    int rcap;
    double* red_part;         // residual-norm partial sums (per block, per right-hand side)
    unsigned* red_tickets;    // per right-hand-side block counters (self-resetting)
    size_t red_cap, ticket_cap;

    int64_t dev_bytes;
    slab_status err;

    // measurement: launch counts per kernel class, optional event timing
    int64_t launches[SLAB_KERNEL_CLASSES];
    int stage1_dense;         // set while the 3-D slab elimination runs (see prof_class)
    int prof_on;
    void* prof;               // ProfRecord (api.cu) while timing is on
};

enum SlabKernelClass {
    KC_COEFF = 0, KC_TREE_FACTOR, KC_ASSEMBLE, KC_PANEL, KC_TRAIL, KC_SYRK, KC_SOLVE_PROD,
    KC_TREE_UP, KC_TREE_DOWN, KC_STENCIL, KC_OTHER,
    KC_SLAB_PANEL, KC_SLAB_TRAIL, KC_SLAB_SYRK      // the same dense kernels inside the 3-D slab elimination
};

// While h->stage1_dense is set (the 3-D slab elimination runs), the dense classes are counted
// under their Stage-1 names, so that the Stage-2 classes time Algorithm 1 alone.
inline int prof_class(const slab_handle* h, int cls) {
    return (h->stage1_dense && (cls == KC_PANEL || cls == KC_TRAIL || cls == KC_SYRK))
               ? cls - KC_PANEL + KC_SLAB_PANEL
               : cls;
}

// Records one launch of class cls on h->stream; with timing on, brackets it by events.
void prof_begin(slab_handle* h, int cls);
void prof_end(slab_handle* h, int cls);
struct ProfScope {
    slab_handle* h;
    int cls;
    ProfScope(slab_handle* hh, int c) : h(hh), cls(c) { prof_begin(h, cls); }
    ~ProfScope() { prof_end(h, cls); }
};
#define SLAB_PROF(h, cls) ProfScope _prof_scope_((h), (cls))
// Further kernel launches made inside one SLAB_PROF scope (split pre-passes, split-K reductions).
inline void prof_extra(slab_handle* h, int cls, int n) { h->launches[prof_class(h, cls)] += n; }

// ---------------------------------------------------------------- tree helpers (host+device)
__host__ __device__ inline int tree_height_count(int s) {
    int H = 0;
    while ((1 << H) <= s) ++H;
    return H;                      // root = 2^(H-1)
}
__host__ __device__ inline int tree_nodes_at(int s, int k) {
    int p = 1 << k;
    return p > s ? 0 : (s - p) / (2 * p) + 1;
}
// height of the right child of node c at height k (-1 if none)
__host__ __device__ inline int tree_right_height(int s, int c, int k) {
    if (k == 0 || c >= s) return -1;
    for (int kk = k - 1; kk >= 0; --kk)
        if (c + (1 << kk) <= s) return kk;
    return -1;
}

// A sizing pass over an arena without memory: buffers are offsets only, so nothing may touch them.
inline bool sizing_pass(const slab_handle* h) { return h->arena && !h->arena->base; }

// ---------------------------------------------------------------- building blocks (api.cu)
// Device allocation of a handle's buffer (from its arena if it has one; counted in dev_bytes).
slab_status slab_dalloc(slab_handle* h, void** p, size_t bytes);
// slab_factor in steps: create validates and allocates every buffer the factor needs (no kernel
// runs); launch enqueues the factor on h->stream with no allocation and no host synchronisation;
// factor_status synchronises the stream and maps the device status word to a slab_status.
slab_status factor_create(const slab_grid* grid, const slab_coeffs* co, int b, const slab_opts* opts,
                          slab_handle** out, SlabArena* arena);
slab_status factor_launch(slab_handle* h, const double* kappa, const double* c);
slab_status factor_status(slab_handle* h);
// Every buffer a solve of k loads needs (solve workspace, FP64 residual, norm reduction).
slab_status solve_prepare(slab_handle* h, int k);
// Zero the self-resetting ticket counters of a handle whose memory may hold another's old data.
slab_status reset_scratch(slab_handle* h);
// u = A^-1 f by one solve pass and `steps` refinement passes, then nrm[q] = ||f_q - A u_q||^2 and
// nrm[k + q] = ||f_q||^2 on the device: enqueued on h->stream, no allocation, no host sync.
slab_status solve_fixed(slab_handle* h, const double* f, double* u, int k, int steps, double* nrm);

// ---------------------------------------------------------------- launchers (defined in .cu files)
// coefficients / stencil (stencil.cu)
slab_status launch_coefficients(slab_handle* h, const double* kappa, const double* c);
slab_status launch_residual(slab_handle* h, const double* u, const double* f, double* r, int k,
                            double* nrm_r, double* nrm_f);   // nrm_* may be NULL (device, k each)
slab_status launch_apply(slab_handle* h, const double* x, double* y, int k);
slab_status launch_boundary_lift(slab_handle* h, const double* g, const double* f, double* fo, int k);
slab_status launch_kappa_gradient(slab_handle* h, const double* u, const double* lam, double* g, int k);
// out = the interface entries of v ([k][N] -> [k][N_I][si], the ABI's interface layout).
slab_status launch_gather_interface(slab_handle* h, const double* v, double* out, int k);
// Sizes the norm-reduction scratch of launch_residual for k right-hand sides.
slab_status ensure_red(slab_handle* h, int k);
// FP64 vector kernels for the Krylov refinement (batched over k vectors of length N)
slab_status vec_dot(slab_handle* h, const double* x, const double* y, int64_t N, int k, double* part, double* out);
slab_status vec_axpy(slab_handle* h, double* y, const double* x, const double* c, double sign, int64_t N, int k);
slab_status vec_scale(slab_handle* h, double* x, const double* nrm2, int64_t N, int k);
slab_status vec_combine(slab_handle* h, double* u, const double* Z, int64_t zstride, const double* c, int j, int k,
                        int64_t N);
size_t vec_dot_part_elems(int k);

// stage 1 (tree.cu)
int tree_kmax();   // right-hand sides per solve-phase launch
size_t tree_down_ws_elems(int s, int m, int NS);
size_t tree_down_tickets(int s, int NS);
template <typename T> slab_status tree_factor(slab_handle* h);
// up pass + reduced load into the interface workspace X, for rhs [r0, r0+K) of F scaled by fscale
template <typename T> slab_status tree_up_gather(slab_handle* h, const double* F, double fscale, int r0, int K);
// down pass from X (interface solution) into U (FP64 [k][N]); accumulate: U += x instead of U = x
template <typename T> slab_status tree_down_scatter(slab_handle* h, double* U, int accumulate, int r0, int K);
template <typename T> slab_status export_ftilde_part(slab_handle* h, double* out, double scale, int r0, int K);
template <typename T> slab_status import_utilde_part(slab_handle* h, const double* in, int r0, int K);

// T assembly (assemble.cu)
template <typename T> slab_status assemble_T(slab_handle* h);

// stage 2 (dense.cu)
template <typename T> slab_status sweep_factor(slab_handle* h);
template <typename T> slab_status sweep_solve(slab_handle* h, int K);
// odd-even elimination order of T (SPD kinds)
int cr_max_batch(int NI);
size_t gj_work_bytes(int s_pad, size_t rsz);
// 3-D slabs
struct Tree3Plan* tree3d_plan(int s, int m, int NS);
void tree3d_plan_free(struct Tree3Plan* P);
int64_t tree3d_nodes(const struct Tree3Plan* P);
int tree3d_mpad(const struct Tree3Plan* P);
int64_t tree3d_zit_elems(const struct Tree3Plan* P);
int64_t tree3d_work_elems(const struct Tree3Plan* P);
int64_t tree3d_xI_elems(const struct Tree3Plan* P);
template <typename T> slab_status tree3d_factor(slab_handle* h);
template <typename T> slab_status tree3d_up_gather(slab_handle* h, const double* F, double fscale, int r0, int K);
template <typename T> slab_status tree3d_down_scatter(slab_handle* h, double* U, int accumulate, int r0, int K);
template <typename T> slab_status tree3d_export(slab_handle* h, double* out, double scale, int r0, int K);
template <typename T> slab_status tree3d_import(slab_handle* h, const double* in, int r0, int K);
// dense building blocks (tensor-core products for FP32, SIMT for FP64); batch > 1 uses strides
template <typename T>
slab_status dense_gemm(slab_handle* h, int cls, int M, int N, int K, T alpha, const T* A, int64_t lda, int64_t sA,
                       const T* B, int64_t ldb, int64_t sB, T beta, T* C, int64_t ldc, int64_t sC, int transC,
                       int lower_only, int batch, int triA = 0);
template <typename T>
slab_status dense_transpose(slab_handle* h, const T* in, int64_t ldin, int64_t sin, T* out, int64_t ldout,
                            int64_t sout, int rows, int cols, int batch);
template <typename T>
slab_status dense_copy(slab_handle* h, const T* in, int64_t sin, T* out, int64_t sout, int64_t n, int batch);
template <typename T>
slab_status dense_tall_cholesky(slab_handle* h, T* W, int ncols, int ident0, int batch, int64_t bstride);
slab_status widen_to_double(slab_handle* h, const float* src, double* dst, int64_t n);
slab_status narrow_to_float(slab_handle* h, const double* src, float* dst, int64_t n);
template <typename T> slab_status cr_factor(slab_handle* h);
template <typename T> slab_status cr_solve(slab_handle* h, int K);

// tensor-core product (tcgemm.cu): C = alpha A B^T + beta C, FP32, A [M][K], B [N][K] row-major
struct TcGemmArgs {
    int M, N, K;
    float alpha, beta;
    const float* A; int64_t lda;
    const float* B; int64_t ldb;
    float* C; int64_t ldc;
    int transC;          // 1: write C^T, i.e. C[col * ldc + row]
    int split;           // 0: plain TF32; 1: 3xTF32; 2: three FP16 products of row-scaled hi/lo splits
                         // (both FP32-level accuracy; 2 needs K % 64 == 0 and the work buffer w16)
    int lower_only;      // skip 128 x BN tiles strictly above the diagonal
    int batch;           // independent products, A/B/C batch strides sA/sB/sC (elements)
    int64_t sA, sB, sC;
    int ksplit;          // > 1: K split over CTAs, partial sums in part[batch][ksplit][M][N] (split 0 / 1)
    float* part;
    void* w16;           // split 2: operand splits and exponents, f16x3_work_bytes(M, N, K, batch, shared)
    size_t w16_bytes;
    int triA = 0;        // splits 0 / 1: 1 A lower triangular (A[m][k] = 0 for k > m), 2 A upper (k < m):
                         // the K range of every 128-row tile is cut to the nonzero part
};
// Work bytes of the split-2 product; shared: B is the first N rows of A (one split serves both).
size_t f16x3_work_bytes(int64_t M, int64_t N, int64_t K, int batch, bool shared);
// True when B can reuse the split of A: same array, strides and batch stride, N <= M.
inline bool f16x3_shared(const TcGemmArgs& g) {
    return g.A == g.B && g.lda == g.ldb && g.sA == g.sB && g.N <= g.M;
}
size_t ozaki_work_bytes(int64_t M, int64_t N, int K);
slab_status ozaki_gemm(cudaStream_t st, int M, int N, int K, double alpha, const double* A, int64_t lda,
                       const double* B, int64_t ldb, double* C, int64_t ldc, int lower_only, void* work,
                       unsigned* err);
// g.split may come back changed (the tuner can run a split-2 request as 3xTF32, split 1).
slab_status tc_gemm(cudaStream_t st, TcGemmArgs& g, unsigned* err);
// Kernels tc_gemm launches besides the product itself: the split-K reduction, the operand splits.
inline int tc_gemm_extra_launches(const TcGemmArgs& g) {
    if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return -1;                 // nothing launched
    return (g.ksplit > 1 ? 1 : 0) + (g.split == 2 ? (f16x3_shared(g) ? 1 : 2) : 0);
}

// Programmatic dependent launch for the chains of short dependent kernels (tall-Cholesky panels,
// their products and pre-passes): a kernel launched with launch_pdl may start while its
// predecessor in the stream is still running; it must call pdl_wait() before it touches anything
// the predecessor writes (the wait returns once the predecessor has completed and its memory is
// visible), and it lets its own dependents start early with pdl_trigger().  Both are no-ops for a
// kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, ((KArgs)args)...);
}

// error helper: latches SLAB_ECUDA in the handle; with SLAB_CUDA_TRACE set in the environment it
// also prints the CUDA error and the source line of the failed call (run with
// CUDA_LAUNCH_BLOCKING=1 to attribute an asynchronous kernel fault to its launch)
slab_status slab_cuda_check(slab_handle* h, cudaError_t e, const char* file, int line);
#define SLAB_CK(h, call)                                                         \
    do {                                                                         \
        cudaError_t _e = (call);                                                 \
        if (_e != cudaSuccess) return slab_cuda_check((h), _e, __FILE__, __LINE__); \
    } while (0)
#define SLAB_CK_LAUNCH(h) SLAB_CK(h, cudaGetLastError())
