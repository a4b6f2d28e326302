// Coefficient setup and the FP64 five-point stencil: residual, apply, kappa gradient.
//
// The operator is the paper's five-point scheme (Sec. 2.1, eq. "discretiation")
// with the operator sign of eq. "var_helm": (A u)_P = n^2 sum_faces k_f (u_P - u_Q)
// + q_P u_P.  These kernels are bound by HBM bandwidth: one coalesced pass over
// u, f and r per right-hand side (the coefficient arrays stay in L2 across
// right-hand sides).
#include <algorithm>

#include "slab_internal.cuh"

namespace {

// CONVECTION (beta = [2][(n+1)^2], velocity x then y): the central first-order term makes the
// couplings direction dependent, AX[P] = -h^2 A[P, P+e_x] = k - beta_x(P) h/2 and
// AXT[P] = -h^2 A[P+e_x, P] = k + beta_x(P+e_x) h/2 (y likewise); the other kinds leave AXT / AYT alone.
__global__ void coeff_kernel(int n, int kind, const double* __restrict__ kappa,
                             const double* __restrict__ c, double omega, const double* __restrict__ beta,
                             double* AX, double* AY, double* DG, double* AXT, double* AYT) {
    const int np1 = n + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x > n) return;
    const int64_t P = (int64_t)y * np1 + x;
    auto face = [&](int64_t a, int64_t b2) -> double {
        return (kind == SLAB_DIFFUSION || kind == SLAB_CONVECTION) ? 0.5 * (kappa[a] + kappa[b2]) : 1.0;
    };
    AX[P] = x < n ? face(P, P + 1) : 0.0;
    AY[P] = y < n ? face(P, P + np1) : 0.0;
    if (kind == SLAB_CONVECTION) {
        const int64_t nodes = (int64_t)np1 * np1;
        const double hh = 0.5 / n;
        const double* bx = beta;
        const double* by = beta + nodes;
        AXT[P] = x < n ? AX[P] + hh * bx[P + 1] : 0.0;
        AYT[P] = y < n ? AY[P] + hh * by[P + np1] : 0.0;
        if (x < n) AX[P] -= hh * bx[P];
        if (y < n) AY[P] -= hh * by[P];
    }
    double d = 0.0;
    if (x >= 1 && x < n && y >= 1 && y < n) {
        d = face(P, P - 1) + face(P, P + 1) + face(P, P - np1) + face(P, P + np1);
        if (kind == SLAB_HELMHOLTZ) {
            const double w = omega / c[P] / n;      // h * omega / c
            d -= w * w;
        }
    }
    DG[P] = d;
}

// r = f - A u (RESID) or y = A u, 2-D, k right-hand sides.  Row P couples to its east / north
// neighbours with -n^2 AX[P], -n^2 AY[P] and to its west / south neighbours with -n^2 AXW[P - e_x],
// -n^2 AYS[P - e_y] (AXW = AX, AYS = AY for the symmetric kinds; the transposed couplings for
// CONVECTION, and the roles swapped for A^T).  Block: 256 threads along x; each
// block covers ST_ROWS grid rows and a group of up to ST_Q right-hand sides (blockIdx.z), so the
// five coefficients of a node are read once per group.
// Norms: each block writes its partial sums of r^2 and f^2 per right-hand side to part; the last
// block of a group (ticket counter) adds the partials in block order, so the sums are deterministic.
constexpr int ST_ROWS = 16;
constexpr int ST_Q = 8;
template <bool RESID, bool NORMF>
__global__ void __launch_bounds__(256) stencil2d_kernel(int n, int k, const double* __restrict__ AX,
                                                        const double* __restrict__ AY,
                                                        const double* __restrict__ AXW,
                                                        const double* __restrict__ AYS,
                                                        const double* __restrict__ DG,
                                                        const double* __restrict__ u,
                                                        const double* __restrict__ f, double* r,
                                                        double* nrm_r, double* nrm_f, double* part,
                                                        unsigned* tickets) {
    const int s = n - 1;
    const int np1 = n + 1;
    const int q0 = blockIdx.z * ST_Q;
    const int nq = min(ST_Q, k - q0);
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1;   // 1..s
    const double n2 = (double)n * (double)n;
    const int64_t N = (int64_t)s * s;
    double rr2[ST_Q], ff2[ST_Q];
#pragma unroll
    for (int q = 0; q < ST_Q; ++q) rr2[q] = ff2[q] = 0.0;
    const int y0 = blockIdx.y * ST_ROWS + 1;
    const int ny = min(ST_ROWS, s - y0 + 1);
    if (x <= s && ny > 0) {
        // per right-hand side a sliding window down this column: wu = row y-1, wc = row y
        double wu[ST_Q], wc[ST_Q];
#pragma unroll
        for (int q = 0; q < ST_Q; ++q) {
            wu[q] = wc[q] = 0.0;
            if (q < nq) {
                const double* uq = u + (q0 + q) * N + (x - 1);
                wu[q] = y0 > 1 ? uq[(int64_t)(y0 - 2) * s] : 0.0;
                wc[q] = uq[(int64_t)(y0 - 1) * s];
            }
        }
        for (int yy = 0; yy < ny; ++yy) {
            const int y = y0 + yy;
            const int64_t P = (int64_t)y * np1 + x;
            const double dg = n2 * DG[P];
            const double aw = x > 1 ? n2 * AXW[P - 1] : 0.0;
            const double ae = x < s ? n2 * AX[P] : 0.0;
            const double as = y > 1 ? n2 * AYS[P - np1] : 0.0;
            const double an = y < s ? n2 * AY[P] : 0.0;
            const int64_t o = (int64_t)(y - 1) * s + (x - 1);
#pragma unroll
            for (int q = 0; q < ST_Q; ++q) {
                if (q < nq) {
                    const double* uq = u + (q0 + q) * N;
                    const double un = y < s ? uq[o + s] : 0.0;
                    const double uw = x > 1 ? uq[o - 1] : 0.0;
                    const double ue = x < s ? uq[o + 1] : 0.0;
                    if (RESID) {
                        // r = f - A u as one chain of five FMAs (the kernel is bound by the FP64 pipe)
                        const double fv = f[(q0 + q) * N + o];
                        double rv = fma(aw, uw, fv);
                        rv = fma(ae, ue, rv);
                        rv = fma(as, wu[q], rv);
                        rv = fma(an, un, rv);
                        rv = fma(-dg, wc[q], rv);
                        r[(q0 + q) * N + o] = rv;
                        rr2[q] += rv * rv;
                        if (NORMF) ff2[q] += fv * fv;
                    } else {
                        r[(q0 + q) * N + o] = dg * wc[q] - aw * uw - ae * ue - as * wu[q] - an * un;
                    }
                    wu[q] = wc[q];
                    wc[q] = un;
                }
            }
        }
    }
    if (!RESID || !nrm_r) return;
    __shared__ double red[2][ST_Q][8];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < ST_Q; ++q) {
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
    if (threadIdx.x < 2 * ST_Q) {
        const int which = threadIdx.x / ST_Q, q = threadIdx.x % ST_Q;
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
            else if (nrm_f) nrm_f[q0 + q] = red2[0];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) tickets[blockIdx.z] = 0;   // ready for the next launch
}

// dL/dkappa_p += -sum_{faces f containing p} (1/2) n^2 (lam_P - lam_Q)(u_P - u_Q), summed over k pairs.
__global__ void kappa_grad2d_kernel(int n, const double* __restrict__ u,
                                    const double* __restrict__ lam, double* g, int k) {
    const int s = n - 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x > n) return;
    const int64_t N = (int64_t)s * s;
    const double c = -0.5 * (double)n * (double)n;
    double acc = 0.0;
    for (int q = 0; q < k; ++q) {
        const double* uq = u + q * N;
        const double* lq = lam + q * N;
        auto val = [&](const double* v, int xx, int yy) -> double {
            return (xx >= 1 && xx <= s && yy >= 1 && yy <= s) ? v[(int64_t)(yy - 1) * s + (xx - 1)] : 0.0;
        };
        const double up = val(uq, x, y), lp = val(lq, x, y);
        const int nx[4] = {x - 1, x + 1, x, x};
        const int ny[4] = {y, y, y - 1, y + 1};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (nx[t] < 0 || nx[t] > n || ny[t] < 0 || ny[t] > n) continue;
            acc += c * (lp - val(lq, nx[t], ny[t])) * (up - val(uq, nx[t], ny[t]));
        }
    }
    g[(int64_t)y * (n + 1) + x] += acc;
}

// ---------------------------------------------------------------- three dimensions
// Seven-point operator on the (n-1)^3 interior nodes, layout [z][y][x]; coefficient arrays over the
// (n+1)^3 nodes: AX / AY / AZ the face toward +x / +y / +z, DG the diagonal, all h^2-scaled.
__global__ void coeff3_kernel(int n, int kind, const double* __restrict__ kappa, double* AX, double* AY, double* AZ,
                              double* DG) {
    const int np1 = n + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    if (x > n) return;
    const int64_t P = ((int64_t)z * np1 + y) * np1 + x;
    const int64_t sy = np1, sz = (int64_t)np1 * np1;
    auto face = [&](int64_t a, int64_t b2) -> double {
        return kind == SLAB_DIFFUSION ? 0.5 * (kappa[a] + kappa[b2]) : 1.0;
    };
    AX[P] = x < n ? face(P, P + 1) : 0.0;
    AY[P] = y < n ? face(P, P + sy) : 0.0;
    AZ[P] = z < n ? face(P, P + sz) : 0.0;
    double d = 0.0;
    if (x >= 1 && x < n && y >= 1 && y < n && z >= 1 && z < n)
        d = face(P, P - 1) + face(P, P + 1) + face(P, P - sy) + face(P, P + sy) + face(P, P - sz) + face(P, P + sz);
    DG[P] = d;
}

// r = f - A u (RESID) or y = A u for k vectors; one thread per x, blockIdx.y = y, blockIdx.z = (z, rhs)
template <bool RESID>
__global__ void __launch_bounds__(128) stencil3d_kernel(int n, int k, const double* __restrict__ AX,
                                                        const double* __restrict__ AY, const double* __restrict__ AZ,
                                                        const double* __restrict__ DG, const double* __restrict__ u,
                                                        const double* __restrict__ f, double* r, int q0) {
    const int s = n - 1, np1 = n + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int y = blockIdx.y + 1;
    const int z = blockIdx.z % s + 1, q = q0 + (int)(blockIdx.z / s);
    if (x > s || q >= k) return;
    const double n2 = (double)n * (double)n;
    const int64_t N = (int64_t)s * s * s;
    const int64_t P = ((int64_t)z * np1 + y) * np1 + x;
    const int64_t o = ((int64_t)(z - 1) * s + (y - 1)) * s + (x - 1);
    const double* uq = u + (int64_t)q * N;
    double Au = DG[P] * uq[o];
    if (x > 1) Au -= AX[P - 1] * uq[o - 1];
    if (x < s) Au -= AX[P] * uq[o + 1];
    if (y > 1) Au -= AY[P - np1] * uq[o - s];
    if (y < s) Au -= AY[P] * uq[o + s];
    if (z > 1) Au -= AZ[P - (int64_t)np1 * np1] * uq[o - (int64_t)s * s];
    if (z < s) Au -= AZ[P] * uq[o + (int64_t)s * s];
    Au *= n2;
    if (RESID) r[(int64_t)q * N + o] = f[(int64_t)q * N + o] - Au;
    else r[(int64_t)q * N + o] = Au;
}

// Dirichlet data into the load: f_out = f + h^-2 sum over the boundary neighbours Q of each
// interior node P of k_PQ g_Q (g over all (n+1)^d nodes per right-hand side, f may be null).
// One thread per interior unknown and right-hand side, x fastest.
__global__ void boundary_lift_kernel(int dim, int n, int k, const double* __restrict__ AX,
                                     const double* __restrict__ AY, const double* __restrict__ AZ,
                                     const double* __restrict__ g, const double* __restrict__ f, double* fo) {
    const int s = n - 1, np1 = n + 1;
    const int64_t N = dim == 3 ? (int64_t)s * s * s : (int64_t)s * s;
    const int64_t nodes = dim == 3 ? (int64_t)np1 * np1 * np1 : (int64_t)np1 * np1;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * k) return;
    const int64_t q = idx / N, o = idx % N;
    const int x = (int)(o % s) + 1;
    const int y = (int)((o / s) % s) + 1;
    const int z = dim == 3 ? (int)(o / ((int64_t)s * s)) + 1 : 0;
    const int64_t P = ((int64_t)z * np1 + y) * np1 + x;
    const int64_t sy = np1, sz = (int64_t)np1 * np1;
    const double* gq = g + q * nodes;
    double v = 0.0;
    if (x == 1) v += AX[P - 1] * gq[P - 1];
    if (x == s) v += AX[P] * gq[P + 1];
    if (y == 1) v += AY[P - sy] * gq[P - sy];
    if (y == s) v += AY[P] * gq[P + sy];
    if (dim == 3) {
        if (z == 1) v += AZ[P - sz] * gq[P - sz];
        if (z == s) v += AZ[P] * gq[P + sz];
    }
    fo[idx] = (f ? f[idx] : 0.0) + (double)n * (double)n * v;
}

// ---------------------------------------------------------------- FP64 vector kernels (Krylov)
// Batched over k vectors of length N, vector q at x + q * N.  Dot products are reduced in a
// fixed order (per-block partials, then one block per vector), so they are deterministic.
constexpr int VD_BLOCKS = 256;

__global__ void __launch_bounds__(256) vdot_partial_kernel(const double* __restrict__ x,
                                                           const double* __restrict__ y, int64_t N,
                                                           double* part) {
    const int q = blockIdx.y;
    x += (int64_t)q * N;
    y += (int64_t)q * N;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
        acc += x[i] * y[i];
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        part[(int64_t)q * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void vdot_final_kernel(const double* __restrict__ part, int nb, double* out) {
    const int q = blockIdx.x;
    __shared__ double red[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(int64_t)q * nb + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = red[0];
}

// y_q += sign * c_q * x_q
__global__ void vaxpy_kernel(double* y, const double* __restrict__ x, const double* __restrict__ c,
                             double sign, int64_t N) {
    const int q = blockIdx.y;
    const double a = sign * c[q];
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
        y[(int64_t)q * N + i] += a * x[(int64_t)q * N + i];
}

// x_q *= 1 / sqrt(nrm2_q)  (left as is when nrm2_q is zero)
__global__ void vscale_kernel(double* x, const double* __restrict__ nrm2, int64_t N) {
    const int q = blockIdx.y;
    const double v = nrm2[q];
    if (!(v > 0.0)) return;
    const double a = 1.0 / sqrt(v);
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < N; i += (int64_t)gridDim.x * 256)
        x[(int64_t)q * N + i] *= a;
}

// u_q += sum_{i < j} c[i][q] Z_i,q   (Z_i at Z + i * zstride)
__global__ void vcombine_kernel(double* u, const double* __restrict__ Z, int64_t zstride,
                                const double* __restrict__ c, int j, int k, int64_t N) {
    const int q = blockIdx.y;
    for (int64_t n = (int64_t)blockIdx.x * 256 + threadIdx.x; n < N; n += (int64_t)gridDim.x * 256) {
        double acc = u[(int64_t)q * N + n];
        for (int i = 0; i < j; ++i) acc += c[(int64_t)i * k + q] * Z[i * zstride + (int64_t)q * N + n];
        u[(int64_t)q * N + n] = acc;
    }
}

}  // namespace

slab_status launch_coefficients(slab_handle* h, const double* kappa, const double* c) {
    const int n = h->n;
    if (h->dim == 3) {
        SLAB_PROF(h, KC_COEFF);
        coeff3_kernel<<<dim3((n + 1 + 127) / 128, n + 1, n + 1), 128, 0, h->stream>>>(n, h->kind, kappa, h->AX, h->AY,
                                                                                    h->AZ, h->DG);
        SLAB_CK_LAUNCH(h);
        return SLAB_OK;
    }
    dim3 grid((n + 1 + 127) / 128, n + 1);
    SLAB_PROF(h, KC_COEFF);
    coeff_kernel<<<grid, 128, 0, h->stream>>>(n, h->kind, kappa, c, h->omega, h->beta, h->AX, h->AY, h->DG, h->AXT,
                                              h->AYT);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status ensure_red(slab_handle* h, int k) {
    const int s = h->n - 1;
    const size_t need = h->dim == 3 ? vec_dot_part_elems(k)
                                    : (size_t)k * ((s + 255) / 256) * ((s + ST_ROWS - 1) / ST_ROWS) * 2;
    const size_t tk = h->dim == 3 ? 0 : (size_t)k;
    if (h->red_cap >= need && h->ticket_cap >= tk) return SLAB_OK;
    if (!h->arena) {
        if (h->red_part) cudaFree(h->red_part);
        if (h->red_tickets) cudaFree(h->red_tickets);
    }
    h->red_part = nullptr; h->red_tickets = nullptr; h->red_cap = h->ticket_cap = 0;
    void* p = nullptr;
    slab_status st = slab_dalloc(h, &p, need * sizeof(double));
    if (st) return st;
    h->red_part = (double*)p;
    h->red_cap = need;
    if (tk) {
        st = slab_dalloc(h, &p, tk * sizeof(unsigned));
        if (st) return st;
        h->red_tickets = (unsigned*)p;
        if (!sizing_pass(h)) SLAB_CK(h, cudaMemsetAsync(h->red_tickets, 0, tk * sizeof(unsigned), h->stream));
        h->ticket_cap = tk;
    }
    return SLAB_OK;
}

namespace {
// East / north and west / south coupling arrays of the 2-D stencil: A's, or A^T's while a
// transposed solve runs (its east coupling is A's west one read from the other end of the face).
struct Couplings { const double *e, *nn, *w, *so; };
Couplings couplings2d(const slab_handle* h) {
    if (!h->AXT) return {h->AX, h->AY, h->AX, h->AY};
    if (h->transposed) return {h->AXT, h->AYT, h->AX, h->AY};
    return {h->AX, h->AY, h->AXT, h->AYT};
}
}  // namespace

slab_status launch_residual(slab_handle* h, const double* u, const double* f, double* r, int k,
                            double* nrm_r, double* nrm_f) {
    const int n = h->n, s = n - 1;
    if (k <= 0) return SLAB_OK;
    if (h->dim == 3) {
        {
            SLAB_PROF(h, KC_STENCIL);
            // gridDim.z = s x (right-hand sides of one launch) stays within 65535
            const int qc = 65535 / s;
            for (int q0 = 0; q0 < k; q0 += qc) {
                const int kq = std::min(qc, k - q0);
                stencil3d_kernel<true><<<dim3((s + 127) / 128, s, s * kq), 128, 0, h->stream>>>(
                    n, q0 + kq, h->AX, h->AY, h->AZ, h->DG, u, f, r, q0);
                SLAB_CK_LAUNCH(h);
            }
            prof_extra(h, KC_STENCIL, (k - 1) / qc);
        }
        if (!nrm_r) return SLAB_OK;
        const slab_status sr = ensure_red(h, k);
        if (sr) return sr;
        const int64_t N = (int64_t)s * s * s;
        slab_status st = vec_dot(h, r, r, N, k, h->red_part, nrm_r);
        if (!st && nrm_f) st = vec_dot(h, f, f, N, k, h->red_part, nrm_f);
        return st;
    }
    dim3 grid((s + 255) / 256, (s + ST_ROWS - 1) / ST_ROWS, (k + ST_Q - 1) / ST_Q);
    double* part = nullptr;
    unsigned* tickets = nullptr;
    if (nrm_r) {
        const slab_status sr = ensure_red(h, k);
        if (sr) return sr;
        part = h->red_part; tickets = h->red_tickets;
    }
    SLAB_PROF(h, KC_STENCIL);
    const Couplings cp = couplings2d(h);
    if (nrm_f)
        stencil2d_kernel<true, true><<<grid, 256, 0, h->stream>>>(n, k, cp.e, cp.nn, cp.w, cp.so, h->DG, u, f, r,
                                                                  nrm_r, nrm_f, part, tickets);
    else
        stencil2d_kernel<true, false><<<grid, 256, 0, h->stream>>>(n, k, cp.e, cp.nn, cp.w, cp.so, h->DG, u, f, r,
                                                                   nrm_r, nullptr, part, tickets);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status launch_boundary_lift(slab_handle* h, const double* g, const double* f, double* fo, int k) {
    const int s = h->n - 1;
    const int64_t tot = (h->dim == 3 ? (int64_t)s * s * s : (int64_t)s * s) * k;
    if (tot <= 0) return SLAB_OK;
    SLAB_PROF(h, KC_OTHER);
    boundary_lift_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, h->stream>>>(h->dim, h->n, k, h->AX, h->AY, h->AZ,
                                                                               g, f, fo);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status launch_apply(slab_handle* h, const double* x, double* y, int k) {
    const int n = h->n, s = n - 1;
    if (k <= 0) return SLAB_OK;
    if (h->dim == 3) {
        SLAB_PROF(h, KC_STENCIL);
        const int qc = 65535 / s;
        for (int q0 = 0; q0 < k; q0 += qc) {
            const int kq = std::min(qc, k - q0);
            stencil3d_kernel<false><<<dim3((s + 127) / 128, s, s * kq), 128, 0, h->stream>>>(
                n, q0 + kq, h->AX, h->AY, h->AZ, h->DG, x, nullptr, y, q0);
            SLAB_CK_LAUNCH(h);
        }
        prof_extra(h, KC_STENCIL, (k - 1) / qc);
        return SLAB_OK;
    }
    dim3 grid((s + 255) / 256, (s + ST_ROWS - 1) / ST_ROWS, (k + ST_Q - 1) / ST_Q);
    SLAB_PROF(h, KC_STENCIL);
    const Couplings cp = couplings2d(h);
    stencil2d_kernel<false, false><<<grid, 256, 0, h->stream>>>(n, k, cp.e, cp.nn, cp.w, cp.so, h->DG, x, nullptr, y,
                                                                nullptr, nullptr, nullptr, nullptr);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

// out[r][q][j] = v[r][interface node (q, j)]: interface q is the plane x = (q + 1) b, its nodes j
// ordered by y (then z), y fastest (the interface-vector layout of the ABI).
__global__ void gather_interface_kernel(int dim, int n, int b, int NI, int k, const double* __restrict__ v,
                                        double* __restrict__ out) {
    const int64_t s = n - 1, si = dim == 3 ? s * s : s, N = dim == 3 ? s * s * s : s * s;
    const int64_t tot = (int64_t)k * NI * si;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e % si, q = (e / si) % NI, r = e / (si * NI);
        const int64_t x = (q + 1) * b;
        const int64_t idx = dim == 3 ? ((j / s) * s + (j % s)) * s + (x - 1) : j * s + (x - 1);
        out[e] = v[r * N + idx];
    }
}

slab_status launch_gather_interface(slab_handle* h, const double* v, double* out, int k) {
    const int64_t tot = (int64_t)k * h->td.NI * h->td.si;
    if (tot <= 0) return SLAB_OK;
    SLAB_PROF(h, KC_OTHER);
    gather_interface_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, 152 * 32), 256, 0, h->stream>>>(
        h->dim, h->n, h->b, h->td.NI, k, v, out);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status launch_kappa_gradient(slab_handle* h, const double* u, const double* lam, double* g, int k) {
    const int n = h->n;
    dim3 grid((n + 1 + 127) / 128, n + 1);
    SLAB_PROF(h, KC_OTHER);
    kappa_grad2d_kernel<<<grid, 128, 0, h->stream>>>(n, u, lam, g, k);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status vec_dot(slab_handle* h, const double* x, const double* y, int64_t N, int k, double* part,
                    double* out) {
    SLAB_PROF(h, KC_OTHER);
    vdot_partial_kernel<<<dim3(VD_BLOCKS, k), 256, 0, h->stream>>>(x, y, N, part);
    SLAB_CK_LAUNCH(h);
    vdot_final_kernel<<<k, 256, 0, h->stream>>>(part, VD_BLOCKS, out);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status vec_axpy(slab_handle* h, double* y, const double* x, const double* c, double sign, int64_t N, int k) {
    SLAB_PROF(h, KC_OTHER);
    vaxpy_kernel<<<dim3(2 * 152, k), 256, 0, h->stream>>>(y, x, c, sign, N);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status vec_scale(slab_handle* h, double* x, const double* nrm2, int64_t N, int k) {
    SLAB_PROF(h, KC_OTHER);
    vscale_kernel<<<dim3(2 * 152, k), 256, 0, h->stream>>>(x, nrm2, N);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status vec_combine(slab_handle* h, double* u, const double* Z, int64_t zstride, const double* c, int j, int k,
                        int64_t N) {
    SLAB_PROF(h, KC_OTHER);
    vcombine_kernel<<<dim3(2 * 152, k), 256, 0, h->stream>>>(u, Z, zstride, c, j, k, N);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

size_t vec_dot_part_elems(int k) { return (size_t)VD_BLOCKS * k; }
