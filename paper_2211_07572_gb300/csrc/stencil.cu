// Coefficient setup and the FP64 five-point stencil: residual, apply, kappa gradient.
//
// The operator is the paper's five-point scheme (Sec. 2.1, eq. "discretiation")
// with the operator sign of eq. "var_helm": (A u)_P = n^2 sum_faces k_f (u_P - u_Q)
// + q_P u_P.  These kernels are bound by HBM bandwidth: one coalesced pass over
// u, f and r per right-hand side (the coefficient arrays stay in L2 across
// right-hand sides).
#include "slab_internal.cuh"

namespace {

__global__ void coeff_kernel(int n, int kind, const double* __restrict__ kappa,
                             const double* __restrict__ c, double omega, double* AX, double* AY,
                             double* DG) {
    const int np1 = n + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x > n) return;
    const int64_t P = (int64_t)y * np1 + x;
    auto face = [&](int64_t a, int64_t b2) -> double {
        return kind == SLAB_DIFFUSION ? 0.5 * (kappa[a] + kappa[b2]) : 1.0;
    };
    AX[P] = x < n ? face(P, P + 1) : 0.0;
    AY[P] = y < n ? face(P, P + np1) : 0.0;
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

// r = f - A u (or y = A x with f == nullptr, sign flipped), 2-D, k right-hand sides.
// Block: 256 threads along x, one grid row per y, blockIdx.z over right-hand-side chunks.
template <bool RESID>
__global__ void __launch_bounds__(256) stencil2d_kernel(int n, const double* __restrict__ AX,
                                                        const double* __restrict__ AY,
                                                        const double* __restrict__ DG,
                                                        const double* __restrict__ u,
                                                        const double* __restrict__ f, double* r,
                                                        int k, int kchunk, double* nrm_r,
                                                        double* nrm_f) {
    const int s = n - 1;
    const int np1 = n + 1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x + 1;   // 1..s
    const int y = blockIdx.y + 1;
    const int r0 = blockIdx.z * kchunk;
    const int r1 = min(k, r0 + kchunk);
    const double n2 = (double)n * (double)n;
    const bool act = x <= s;
    double dg = 0, aw = 0, ae = 0, as = 0, an = 0;
    if (act) {
        const int64_t P = (int64_t)y * np1 + x;
        dg = DG[P];
        aw = AX[P - 1];
        ae = AX[P];
        as = AY[P - np1];
        an = AY[P];
    }
    __shared__ double red[2][8];
    const int64_t N = (int64_t)s * s;
    for (int q = r0; q < r1; ++q) {
        double rr = 0.0, ff = 0.0;
        if (act) {
            const double* uq = u + q * N;
            const int64_t i = (int64_t)(y - 1) * s + (x - 1);
            const double uc = uq[i];
            const double uw = x > 1 ? uq[i - 1] : 0.0;
            const double ue = x < s ? uq[i + 1] : 0.0;
            const double us = y > 1 ? uq[i - s] : 0.0;
            const double un = y < s ? uq[i + s] : 0.0;
            const double Au = n2 * (dg * uc - aw * uw - ae * ue - as * us - an * un);
            if (RESID) {
                const double fv = f[q * N + i];
                rr = fv - Au;
                ff = fv;
                r[q * N + i] = rr;
            } else {
                r[q * N + i] = Au;
            }
        }
        if (RESID && nrm_r) {
            double a = rr * rr, b = ff * ff;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
            }
            const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
            if (l == 0) { red[0][w] = a; red[1][w] = b; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double sa = 0, sb = 0;
                for (int t = 0; t < 8; ++t) { sa += red[0][t]; sb += red[1][t]; }
                atomicAdd(nrm_r + q, sa);
                if (nrm_f) atomicAdd(nrm_f + q, sb);
            }
            __syncthreads();
        }
    }
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

}  // namespace

slab_status launch_coefficients(slab_handle* h, const double* kappa, const double* c) {
    const int n = h->n;
    dim3 grid((n + 1 + 127) / 128, n + 1);
    coeff_kernel<<<grid, 128, 0, h->stream>>>(n, h->kind, kappa, c, h->omega, h->AX, h->AY, h->DG);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

static int kchunk_for(int k) { return k <= 8 ? k : 8; }

slab_status launch_residual(slab_handle* h, const double* u, const double* f, double* r, int k,
                            double* nrm_r, double* nrm_f) {
    const int n = h->n, s = n - 1;
    if (k <= 0) return SLAB_OK;
    const int kc = kchunk_for(k);
    dim3 grid((s + 255) / 256, s, (k + kc - 1) / kc);
    stencil2d_kernel<true><<<grid, 256, 0, h->stream>>>(n, h->AX, h->AY, h->DG, u, f, r, k, kc,
                                                        nrm_r, nrm_f);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status launch_apply(slab_handle* h, const double* x, double* y, int k) {
    const int n = h->n, s = n - 1;
    if (k <= 0) return SLAB_OK;
    const int kc = kchunk_for(k);
    dim3 grid((s + 255) / 256, s, (k + kc - 1) / kc);
    stencil2d_kernel<false><<<grid, 256, 0, h->stream>>>(n, h->AX, h->AY, h->DG, x, nullptr, y, k,
                                                         kc, nullptr, nullptr);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}

slab_status launch_kappa_gradient(slab_handle* h, const double* u, const double* lam, double* g, int k) {
    const int n = h->n;
    dim3 grid((n + 1 + 127) / 128, n + 1);
    kappa_grad2d_kernel<<<grid, 128, 0, h->stream>>>(n, u, lam, g, k);
    SLAB_CK_LAUNCH(h);
    return SLAB_OK;
}
