/*
 * CPU FP64 oracle for the slab factor+solve path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may call
 * this library.  It shares no code with the CUDA path.
 *
 * What it computes is the plain definition of the problem the slab method
 * solves exactly (up to rounding): u = A^{-1} f for the finite-difference
 * matrix A, by
 *   - sparse (CSR) assembly of A from the stencil,
 *   - a banded LU in the natural ordering (x fastest) with half-bandwidth
 *     w = (n-1)^(d-1), without pivoting for the SPD kinds and with partial
 *     pivoting (pivot = first row of largest |a_ik|) for Helmholtz,
 *   - forward/back substitution and an FP64 residual.
 * A naive dense LU with partial pivoting (separate code) serves as the
 * brute-force check of the banded one on tiny grids.
 *
 * Operator (the paper's five-point scheme, Sec. 2.1 eq. "discretiation", with the
 * sign of the operator A = -Lap - kappa^2 b of eq. "var_helm", Sec. 1.1):
 *   (A u)_P = h^-2 sum_{faces P~Q} k_PQ (u_P - u_Q) + q_P u_P,   u_Q = 0 on the boundary,
 * k_PQ = (kappa_P + kappa_Q)/2 for diffusion, 1 for Poisson and Helmholtz;
 * q_P = 0, except Helmholtz where q_P = -(omega / c_P)^2.
 * Convection-diffusion (a second-order elliptic operator with a first-order term, the broad
 * operator class of Sec. 1.1, eq. "bvp"): -div(kappa grad u) + beta . grad u, the first-order
 * term by central differences at P,
 *   (A u)_P += sum_a beta_a(P) (u_{P+e_a} - u_{P-e_a}) / (2h),
 * so the entry of row P at the neighbour Q = P + s e_a (s = +-1) is -h^-2 k_PQ + s beta_a(P)/(2h)
 * and A is not symmetric.
 * Node fields are given at all (n+1)^d nodes, C order [z][y][x].
 *
 * Gradient (adjoint of the loss L(u(kappa))): for the diffusion and convection kinds (the
 * first-order term does not depend on kappa),
 *   dL/dkappa_p = -sum_{faces f containing p} (1/2) h^-2 (lam_P - lam_Q)(u_P - u_Q),
 * with boundary values of lam and u equal to zero, since d k_f / d kappa_p = 1/2
 * and dA/dk_f = h^-2 (e_P - e_Q)(e_P - e_Q)^T; lam solves A^T lam = dL/du.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_POISSON 0
#define ORC_DIFFUSION 1
#define ORC_HELMHOLTZ 2
#define ORC_CONVECTION 3

static int64_t ipow(int64_t a, int e) { int64_t r = 1; while (e-- > 0) r *= a; return r; }

/* node index in the (n+1)^d node array for interior/boundary coordinates */
static int64_t node_id(int dim, int n, int x, int y, int z) {
    int64_t np1 = n + 1;
    return dim == 2 ? (int64_t)y * np1 + x : ((int64_t)z * np1 + y) * np1 + x;
}

static double face_coef(int kind, const double* kappa, int64_t p, int64_t q) {
    if (kind == ORC_DIFFUSION || kind == ORC_CONVECTION) return 0.5 * (kappa[p] + kappa[q]);
    return 1.0;
}

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Number of stored entries of the assembled matrix (upper bound used for allocation). */
int64_t orc_nnz_bound(int dim, int n) {
    return ipow(n - 1, dim) * (2 * dim + 1);
}

/*
 * CSR assembly of A.  rowptr has N+1 entries; col/val have orc_nnz_bound entries.
 * Columns within a row are sorted ascending.  Returns nnz.  beta ([dim][(n+1)^d], the velocity
 * components x, y(, z) at the nodes) is read for the convection kind only.
 */
int64_t orc_assemble(int dim, int n, int kind, const double* kappa, const double* c,
                     double omega, const double* beta, int64_t* rowptr, int64_t* col, double* val) {
    const int m = n - 1;
    const int64_t nodes = ipow(n + 1, dim);
    const double ih2 = (double)n * (double)n;
    const int zmax = dim == 3 ? m : 1;
    int64_t nnz = 0, row = 0;
    rowptr[0] = 0;
    for (int z = 1; z <= zmax; ++z)
        for (int y = 1; y <= m; ++y)
            for (int x = 1; x <= m; ++x, ++row) {
                const int zz = dim == 3 ? z : 0;
                int64_t P = node_id(dim, n, x, y, zz);
                /* neighbour offsets in sorted column order: -z, -y, -x, 0, +x, +y, +z */
                int nx[7], ny[7], nz[7], cnt = 0;
                if (dim == 3) { nx[cnt] = x; ny[cnt] = y; nz[cnt] = zz - 1; ++cnt; }
                nx[cnt] = x; ny[cnt] = y - 1; nz[cnt] = zz; ++cnt;
                nx[cnt] = x - 1; ny[cnt] = y; nz[cnt] = zz; ++cnt;
                int self = cnt; nx[cnt] = x; ny[cnt] = y; nz[cnt] = zz; ++cnt;
                nx[cnt] = x + 1; ny[cnt] = y; nz[cnt] = zz; ++cnt;
                nx[cnt] = x; ny[cnt] = y + 1; nz[cnt] = zz; ++cnt;
                if (dim == 3) { nx[cnt] = x; ny[cnt] = y; nz[cnt] = zz + 1; ++cnt; }
                double diag = 0.0;
                for (int t = 0; t < cnt; ++t) {
                    if (t == self) continue;
                    int64_t Q = node_id(dim, n, nx[t], ny[t], nz[t]);
                    diag += ih2 * face_coef(kind, kappa, P, Q);
                }
                if (kind == ORC_HELMHOLTZ) {
                    double w = omega / c[P];
                    diag -= w * w;
                }
                for (int t = 0; t < cnt; ++t) {
                    int bx = nx[t], by = ny[t], bz = nz[t];
                    if (t == self) {
                        col[nnz] = row; val[nnz] = diag; ++nnz; continue;
                    }
                    int interior = bx >= 1 && bx <= m && by >= 1 && by <= m &&
                                   (dim == 2 || (bz >= 1 && bz <= m));
                    if (!interior) continue;     /* Dirichlet node: eliminated */
                    int64_t Q = node_id(dim, n, bx, by, bz);
                    int64_t qrow = dim == 2 ? (int64_t)(by - 1) * m + (bx - 1)
                                            : ((int64_t)(bz - 1) * m + (by - 1)) * m + (bx - 1);
                    double v = -ih2 * face_coef(kind, kappa, P, Q);
                    if (kind == ORC_CONVECTION) {
                        /* direction a and sign s of Q - P; beta_a(P) s / (2h) */
                        const int dx = bx - x, dy = by - y, dz = bz - zz;
                        const int a = dx ? 0 : (dy ? 1 : 2);
                        const int sgn = dx + dy + dz;
                        v += 0.5 * (double)n * (double)sgn * beta[(int64_t)a * nodes + P];
                    }
                    col[nnz] = qrow;
                    val[nnz] = v;
                    ++nnz;
                }
                rowptr[row + 1] = nnz;
            }
    return nnz;
}

/*
 * Dirichlet data moved into the load (the problem of Sec. 1.1 with u = g on the boundary):
 * eliminating the boundary unknowns from the interior rows of the full operator gives
 *   A u_I = f_I + h^-2 sum_{faces P~Q, Q on the boundary} k_PQ g_Q,
 * so f_out[r][P] = f[r][P] + that sum (f may be NULL: zero).  g is [k][(n+1)^d] over all nodes
 * (interior entries unused), f and f_out are [k][(n-1)^d] in the natural interior order.
 */
void orc_boundary_lift(int dim, int n, int kind, const double* kappa, int k, const double* g,
                       const double* f, double* f_out) {
    const int m = n - 1;
    const double ih2 = (double)n * (double)n;
    const int zmax = dim == 3 ? m : 1;
    const int64_t N = ipow(m, dim), nodes = ipow(n + 1, dim);
    for (int r = 0; r < k; ++r) {
        const double* gr = g + (int64_t)r * nodes;
        int64_t row = 0;
        for (int z = 1; z <= zmax; ++z)
            for (int y = 1; y <= m; ++y)
                for (int x = 1; x <= m; ++x, ++row) {
                    const int zz = dim == 3 ? z : 0;
                    const int64_t P = node_id(dim, n, x, y, zz);
                    int nx[6], ny[6], nz[6], cnt = 0;
                    nx[cnt] = x - 1; ny[cnt] = y; nz[cnt] = zz; ++cnt;
                    nx[cnt] = x + 1; ny[cnt] = y; nz[cnt] = zz; ++cnt;
                    nx[cnt] = x; ny[cnt] = y - 1; nz[cnt] = zz; ++cnt;
                    nx[cnt] = x; ny[cnt] = y + 1; nz[cnt] = zz; ++cnt;
                    if (dim == 3) {
                        nx[cnt] = x; ny[cnt] = y; nz[cnt] = zz - 1; ++cnt;
                        nx[cnt] = x; ny[cnt] = y; nz[cnt] = zz + 1; ++cnt;
                    }
                    double v = f ? f[(int64_t)r * N + row] : 0.0;
                    for (int t = 0; t < cnt; ++t) {
                        const int bx = nx[t], by = ny[t], bz = nz[t];
                        const int interior = bx >= 1 && bx <= m && by >= 1 && by <= m &&
                                             (dim == 2 || (bz >= 1 && bz <= m));
                        if (interior) continue;
                        const int64_t Q = node_id(dim, n, bx, by, bz);
                        v += ih2 * face_coef(kind, kappa, P, Q) * gr[Q];
                    }
                    f_out[(int64_t)r * N + row] = v;
                }
    }
}

/* y = A x for k vectors (x, y laid out [k][N]). */
void orc_csr_matvec(int64_t N, const int64_t* rowptr, const int64_t* col, const double* val,
                    int k, const double* x, double* y) {
    for (int r = 0; r < k; ++r) {
        const double* xr = x + (int64_t)r * N;
        double* yr = y + (int64_t)r * N;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            double s = 0.0;
            for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) s += val[t] * xr[col[t]];
            yr[i] = s;
        }
    }
}

/*
 * Banded storage, column major: column j holds rows j-ku .. j+kl, entry
 * A(i,j) at ab[j*ld + (ku + i - j)], ld = kl + ku + 1.  With pivoting the
 * caller gives ku = 2w so the fill created by row interchanges fits.
 */
int64_t orc_band_ld(int64_t w, int pivot) { return pivot ? 3 * w + 1 : 2 * w + 1; }

void orc_band_from_csr(int64_t N, int64_t w, int pivot, const int64_t* rowptr,
                       const int64_t* col, const double* val, double* ab) {
    const int64_t ku = pivot ? 2 * w : w, ld = orc_band_ld(w, pivot);
    memset(ab, 0, sizeof(double) * (size_t)(N * ld));
    for (int64_t i = 0; i < N; ++i)
        for (int64_t t = rowptr[i]; t < rowptr[i + 1]; ++t) {
            int64_t j = col[t];
            ab[j * ld + (ku + i - j)] = val[t];
        }
}

/*
 * In-place banded LU.  pivot = 0: no interchanges (SPD kinds).  pivot = 1:
 * partial pivoting within the kl = w subdiagonals (first largest |.| wins).
 * ipiv[j] = row swapped with row j.  Returns 0, or j+1 if U(j,j) == 0.
 */
int orc_band_lu(int64_t N, int64_t w, int pivot, double* ab, int64_t* ipiv) {
    const int64_t kl = w, ku = pivot ? 2 * w : w, ld = orc_band_ld(w, pivot);
#define AB(i, j) ab[(j) * ld + (ku + (i) - (j))]
    int info = 0;
    for (int64_t k = 0; k < N; ++k) {
        const int64_t ilast = k + kl < N - 1 ? k + kl : N - 1;
        int64_t p = k;
        if (pivot) {
            double best = fabs(AB(k, k));
            for (int64_t i = k + 1; i <= ilast; ++i)
                if (fabs(AB(i, k)) > best) { best = fabs(AB(i, k)); p = i; }
        }
        ipiv[k] = p;
        const int64_t jlast = k + ku < N - 1 ? k + ku : N - 1;
        if (p != k)
            for (int64_t j = k; j <= jlast; ++j) {
                double t = AB(k, j); AB(k, j) = AB(p, j); AB(p, j) = t;
            }
        const double piv = AB(k, k);
        if (piv == 0.0) { if (!info) info = (int)(k + 1); continue; }
        const double rp = 1.0 / piv;
        for (int64_t i = k + 1; i <= ilast; ++i) AB(i, k) *= rp;
        /* rank-1 update of the trailing band window; columns are independent */
#pragma omp parallel for schedule(static) if (jlast - k > 256)
        for (int64_t j = k + 1; j <= jlast; ++j) {
            const double ukj = AB(k, j);
            if (ukj == 0.0) continue;
            double* cj = &AB(k + 1, j);
            const double* lk = &AB(k + 1, k);
            for (int64_t i = 0; i < ilast - k; ++i) cj[i] -= lk[i] * ukj;
        }
    }
#undef AB
    return info;
}

/* Solve with the banded LU for k right-hand sides laid out [k][N] (in place). */
void orc_band_solve(int64_t N, int64_t w, int pivot, const double* ab, const int64_t* ipiv,
                    int k, double* x) {
    const int64_t kl = w, ku = pivot ? 2 * w : w, ld = orc_band_ld(w, pivot);
#define AB(i, j) ab[(j) * ld + (ku + (i) - (j))]
#pragma omp parallel for schedule(dynamic) if (k > 1)
    for (int r = 0; r < k; ++r) {
        double* b = x + (int64_t)r * N;
        for (int64_t j = 0; j < N; ++j) {            /* L y = P b */
            int64_t p = ipiv[j];
            if (p != j) { double t = b[j]; b[j] = b[p]; b[p] = t; }
            const double bj = b[j];
            const int64_t ilast = j + kl < N - 1 ? j + kl : N - 1;
            for (int64_t i = j + 1; i <= ilast; ++i) b[i] -= AB(i, j) * bj;
        }
        for (int64_t j = N - 1; j >= 0; --j) {       /* U x = y */
            b[j] /= AB(j, j);
            const double bj = b[j];
            const int64_t ifirst = j - ku > 0 ? j - ku : 0;
            for (int64_t i = ifirst; i < j; ++i) b[i] -= AB(i, j) * bj;
        }
    }
#undef AB
}

/*
 * Naive dense LU with partial pivoting, row-major a[N][N], solving for k
 * right-hand sides b[k][N] in place.  Brute-force check for tiny grids.
 */
int orc_dense_solve(int64_t N, double* a, int k, double* b) {
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    for (int64_t i = 0; i < N; ++i) perm[i] = i;
    int info = 0;
    for (int64_t c = 0; c < N; ++c) {
        int64_t p = c;
        for (int64_t i = c + 1; i < N; ++i)
            if (fabs(a[i * N + c]) > fabs(a[p * N + c])) p = i;
        if (p != c) {
            for (int64_t j = 0; j < N; ++j) { double t = a[c * N + j]; a[c * N + j] = a[p * N + j]; a[p * N + j] = t; }
            int64_t t = perm[c]; perm[c] = perm[p]; perm[p] = t;
        }
        if (a[c * N + c] == 0.0) { info = (int)(c + 1); continue; }
        for (int64_t i = c + 1; i < N; ++i) {
            double l = a[i * N + c] / a[c * N + c];
            a[i * N + c] = l;
            for (int64_t j = c + 1; j < N; ++j) a[i * N + j] -= l * a[c * N + j];
        }
    }
    double* y = (double*)malloc(sizeof(double) * (size_t)N);
    for (int r = 0; r < k; ++r) {
        double* br = b + (int64_t)r * N;
        for (int64_t i = 0; i < N; ++i) y[i] = br[perm[i]];
        for (int64_t i = 0; i < N; ++i)
            for (int64_t j = 0; j < i; ++j) y[i] -= a[i * N + j] * y[j];
        for (int64_t i = N - 1; i >= 0; --i) {
            for (int64_t j = i + 1; j < N; ++j) y[i] -= a[i * N + j] * y[j];
            y[i] /= a[i * N + i];
        }
        memcpy(br, y, sizeof(double) * (size_t)N);
    }
    free(y);
    free(perm);
    return info;
}

/*
 * Gradient of a loss with respect to the node coefficients kappa of the
 * diffusion operator, given the state u and the adjoint lam (both [N]).
 * g has (n+1)^d entries (boundary nodes included).
 */
void orc_kappa_gradient(int dim, int n, const double* u, const double* lam, double* g) {
    const int m = n - 1;
    const int64_t np1 = n + 1;
    const double ih2 = (double)n * (double)n;
    const int64_t nodes = ipow(np1, dim);
    memset(g, 0, sizeof(double) * (size_t)nodes);
    const int zlo = dim == 3 ? 0 : 0, zhi = dim == 3 ? n : 0;
    /* value of an interior vector at node (x,y,z); zero on the boundary */
#define VAL(v, x, y, z) (((x) < 1 || (x) > m || (y) < 1 || (y) > m || (dim == 3 && ((z) < 1 || (z) > m))) ? 0.0 \
        : (v)[dim == 2 ? (int64_t)((y) - 1) * m + ((x) - 1) : ((int64_t)((z) - 1) * m + ((y) - 1)) * m + ((x) - 1)])
    for (int z = zlo; z <= zhi; ++z)
        for (int y = 0; y <= n; ++y)
            for (int x = 0; x <= n; ++x) {
                /* faces from (x,y,z) in the +x, +y, +z directions */
                for (int a = 0; a < dim; ++a) {
                    int x2 = x + (a == 0), y2 = y + (a == 1), z2 = z + (a == 2);
                    if (x2 > n || y2 > n || (dim == 3 && z2 > n)) continue;
                    /* a face between two boundary nodes carries no unknown */
                    double du = VAL(u, x, y, z) - VAL(u, x2, y2, z2);
                    double dl = VAL(lam, x, y, z) - VAL(lam, x2, y2, z2);
                    double contrib = -0.5 * ih2 * dl * du;
                    g[node_id(dim, n, x, y, z)] += contrib;
                    g[node_id(dim, n, x2, y2, z2)] += contrib;
                }
            }
#undef VAL
}
