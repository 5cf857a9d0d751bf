// Set-up, normalisation, misfit, gradient and adjoint-basis kernels.
#include <algorithm>

#include "csem_internal.cuh"
#include "csem_td.cuh"
#include "csem_es.cuh"

namespace csem {

// ---------------------------------------------------------------------------
// rho (cells) -> dt/eps on every E edge, eps = sigma_e / (2 w0)  (Sec. 2, Eq. 2)
// sigma_e = sum_c V_c / rho_c / sum_c V_c over the (up to four) cells sharing e.
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_coef_init(const GeoD g, const R *__restrict__ rho, const R *__restrict__ rho_z,
                            R *__restrict__ cE, double two_w0_dt, int *bad) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (t >= g.vol) return;
    const int i = (int)(t % g.pitch);
    const long long r = t / g.pitch;
    const int j = (int)(r % g.NY);
    const int k = (int)(r / g.NY);
    double num = 0.0, den = 0.0;
    // cell offsets for each component: Ex spans (j-1..j, k-1..k) at cell column i, etc.
    int i0 = i, i1 = i, j0 = j, j1 = j, k0 = k, k1 = k;
    bool on = false;
    if (c == 0) { on = (i < g.nx); j0 = j - 1; k0 = k - 1; }
    if (c == 1) { on = (j < g.ny); i0 = i - 1; k0 = k - 1; }
    if (c == 2) { on = (k < g.nz); i0 = i - 1; j0 = j - 1; }
    R out = R(0);
    if (on && i < g.NX) {
        for (int kk = k0; kk <= k1; ++kk)
            for (int jj = j0; jj <= j1; ++jj)
                for (int ii = i0; ii <= i1; ++ii) {
                    if (ii < 0 || jj < 0 || kk < 0 || ii >= g.nx || jj >= g.ny || kk >= g.nz) continue;
                    const double V = g.hx[ii] * g.hy[jj] * g.hz[kk];
                    const double rc = (double)(c == 2 ? rho_z : rho)[((long long)kk * g.ny + jj) * g.nx + ii];
                    if (!(rc > 0.0) || !isfinite(rc)) atomicOr(bad, 1);
                    num += V / rc;
                    den += V;
                }
        if (den > 0.0 && num > 0.0) out = (R)(two_w0_dt * den / num);
    }
    cE[(long long)c * g.vol + t] = out;
}

template <typename R>
cudaError_t launch_coef_init(const GeoD &g, const R *rho, const R *rho_z, R *cE, double two_w0_dt, int *bad,
                             cudaStream_t st) {
    dim3 grid((unsigned)((g.vol + 255) / 256), 3);
    k_coef_init<R><<<grid, 256, 0, st>>>(g, rho, rho_z, cE, two_w0_dt, bad);
    g_launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// normalisation of volumes: out = alpha_k * (acc - comp)   (Sec. 2, Eq. 3)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_finalize_volume(typename C2<R>::T *acc, const typename C2<R>::T *comp, long long vol, int S,
                                  int nf, const double2 *alpha) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= vol) return;
    const int sc = blockIdx.y;           // s*3 + c
    for (int f = 0; f < nf; ++f) {
        const long long o = ((long long)sc * nf + f) * vol + t;
        typename C2<R>::T a = acc[o];
        double ar = a.x, ai = a.y;
        if (comp) { ar -= comp[o].x; ai -= comp[o].y; }
        const double2 al = alpha[f];
        a.x = (R)(al.x * ar - al.y * ai);
        a.y = (R)(al.x * ai + al.y * ar);
        acc[o] = a;
    }
}

template <typename R>
cudaError_t launch_finalize_volume(typename C2<R>::T *acc, const typename C2<R>::T *comp, long long vol, int S,
                                   int nf, const double2 *alpha, cudaStream_t st) {
    dim3 grid((unsigned)((vol + 255) / 256), (unsigned)(S * 3));
    k_finalize_volume<R><<<grid, 256, 0, st>>>(acc, comp, vol, S, nf, alpha);
    g_launches++;
    return cudaGetLastError();
}

__global__ void k_finalize_receivers(const double2 *racc, double *out, int n, int nf, const double2 *alpha) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double2 a = racc[t], al = alpha[t % nf];
    out[2 * t] = al.x * a.x - al.y * a.y;
    out[2 * t + 1] = al.x * a.y + al.y * a.x;
}

cudaError_t launch_finalize_receivers(const double2 *racc, double *out, int S, int n_rec, int nf,
                                      const double2 *alpha, cudaStream_t st) {
    const int n = S * n_rec * nf;
    if (n == 0) return cudaSuccess;
    k_finalize_receivers<<<(n + 255) / 256, 256, 0, st>>>(racc, out, n, nf, alpha);
    g_launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// adjoint series coefficients: c_k = k_k conj(r_k) / dt -> [Re c; Im c]  (Sec. 3.2-3.3)
// ---------------------------------------------------------------------------
__global__ void k_adjoint_coef(const double *resid, double *coef, int n, int nf, const double2 *kf, double inv_dt) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;   // (s, r, f)
    if (t >= n) return;
    const int f = t % nf;
    const int sr = t / nf;
    const double rr = resid[2 * t], ri = -resid[2 * t + 1];   // conj(r)
    const double2 k = kf[f];
    coef[(long long)sr * 2 * nf + f] = (k.x * rr - k.y * ri) * inv_dt;
    coef[(long long)sr * 2 * nf + nf + f] = (k.x * ri + k.y * rr) * inv_dt;
}

cudaError_t launch_adjoint_coef(const double *resid, double *coef, int S, int n_rec, int nf, const double2 *kf,
                                double inv_dt, cudaStream_t st) {
    const int n = S * n_rec * nf;
    k_adjoint_coef<<<(n + 255) / 256, 256, 0, st>>>(resid, coef, n, nf, kf, inv_dt);
    g_launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// gradient (Sec. 3.1 isotropic form, Sec. 3.5 chain rule)
//   edge:  p_e = -Re sum_s sum_k conj(v)_{e,k} E_{e,k}
//   cell:  dphi/dsigma_c = V_c / 4 * sum of p_e over the 12 edges of c
// (dV_e / sum_{c at e} V_c = 1/4 on every edge that carries a field; the
// outer-boundary edges hold E = 0.)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_grad_edge(const typename C2<R>::T *E, const typename C2<R>::T *V, long long vol, int S, int nf,
                            R *pe) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (t >= vol) return;
    double acc = 0.0;
    for (int s = 0; s < S; ++s)
        for (int f = 0; f < nf; ++f) {
            const long long o = (((long long)s * 3 + c) * nf + f) * vol + t;
            const typename C2<R>::T e = E[o], v = V[o];
            acc += (double)v.x * (double)e.x - (double)v.y * (double)e.y;
        }
    pe[(long long)c * vol + t] = (R)(-acc);
}

// rho_v, grad_v non-null: VTI, the x and y edges feed grad (sigma_h), the z edges grad_v (sigma_v)
template <typename R>
__global__ void k_grad_cell(const GeoD g, const R *pe, const R *rho, const R *rho_v, int wrt, R *grad, R *grad_v) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long cells = (long long)g.nx * g.ny * g.nz;
    if (t >= cells) return;
    const int i = (int)(t % g.nx);
    const long long r = t / g.nx;
    const int j = (int)(r % g.ny);
    const int k = (int)(r / g.ny);
    const R *px = pe, *py = pe + g.vol, *pz = pe + 2 * g.vol;
    auto at = [&](int ii, int jj, int kk) { return ((long long)kk * g.NY + jj) * g.pitch + ii; };
    double sh = 0.0, sv = 0.0;
    for (int d1 = 0; d1 < 2; ++d1)
        for (int d0 = 0; d0 < 2; ++d0) {
            sh += (double)px[at(i, j + d0, k + d1)];
            sh += (double)py[at(i + d0, j, k + d1)];
            sv += (double)pz[at(i + d0, j + d1, k)];
        }
    const double V = g.hx[i] * g.hy[j] * g.hz[k];
    if (grad_v) {
        double gh = 0.25 * V * sh, gv = 0.25 * V * sv;   // d phi / d sigma_h, d phi / d sigma_v
        if (wrt == 1) { gh = -gh / (double)rho[t]; gv = -gv / (double)rho_v[t]; }
        grad[t] += (R)gh;
        grad_v[t] += (R)gv;
        return;
    }
    double gs = 0.25 * V * (sh + sv);           // d phi / d sigma_c
    if (wrt == 1) gs = -gs / (double)rho[t];    // d phi / d ln rho_c = -sigma_c d phi / d sigma_c
    grad[t] += (R)gs;
}

template <typename R>
cudaError_t launch_gradient(const GeoD &g, const R *rho, const typename C2<R>::T *E, const typename C2<R>::T *V,
                            int S, int nf, int wrt, bool vti, R *edge_scratch, R *grad, cudaStream_t st) {
    dim3 ge((unsigned)((g.vol + 255) / 256), 3);
    k_grad_edge<R><<<ge, 256, 0, st>>>(E, V, g.vol, S, nf, edge_scratch);
    const long long cells = (long long)g.nx * g.ny * g.nz;
    k_grad_cell<R><<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(g, edge_scratch, rho, vti ? rho + cells : nullptr,
                                                                      wrt, grad, vti ? grad + cells : nullptr);
    g_launches += 2;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_grad_cells(const GeoD &g, const R *rho, const R *pe, int wrt, bool vti, R *grad, cudaStream_t st) {
    const long long cells = (long long)g.nx * g.ny * g.nz;
    k_grad_cell<R><<<(unsigned)((cells + 255) / 256), 256, 0, st>>>(g, pe, rho, vti ? rho + cells : nullptr, wrt,
                                                                      grad, vti ? grad + cells : nullptr);
    g_launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// early end of a forward data run: convergence of the running receiver transform
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_es_check(const double2 *racc, double2 *prev, double2 *fin, int n,
                                                  double tol, int chunk, int last, int steps_at, int *state) {
    __shared__ int moved;
    if (state[0]) return;                      // already ended: the kept spectra stay
    if (threadIdx.x == 0) moved = (chunk == 0) ? 1 : 0;
    __syncthreads();
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double2 a = racc[t], b = prev[t];
        const double dr = a.x - b.x, di = a.y - b.y;
        if (sqrt(dr * dr + di * di) > tol * sqrt(a.x * a.x + a.y * a.y)) moved = 1;
    }
    __syncthreads();
    const bool done = !moved || last;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double2 a = racc[t];
        prev[t] = a;
        if (done) fin[t] = a;
    }
    if (done && threadIdx.x == 0) {
        state[1] = steps_at;
        state[0] = 1;
    }
}

cudaError_t launch_es_check(const double2 *racc, double2 *prev, double2 *fin, int n, double tol, int chunk,
                            int last, int steps_at, int *state, cudaStream_t st) {
    k_es_check<<<1, 256, 0, st>>>(racc, prev, fin, n, tol, chunk, last, steps_at, state);
    g_launches++;
    return cudaGetLastError();
}

template <typename R>
__global__ void __launch_bounds__(256) k_es_vol_stats(const typename C2<R>::T *acc, typename C2<R>::T *prev,
                                                      long long vol, int nf, float tol, float floor_frac,
                                                      EsTail tail, unsigned *stats) {
    const int blk = blockIdx.y;                       // (s*3 + c)*nf + f
    const int f = blk % nf;
    const long long base = (long long)blk * vol;
    // entries below floor_frac of the frequency's largest magnitude at the previous check are
    // held to an absolute bound (the decision is taken in FP32)
    const float floor_a = floor_frac * __uint_as_float(stats[2 * nf + f]);
    const float tf = tail.f[f];                       // remainder per unit change (geometric tail)
    float amax = 0.f;
    unsigned viol = 0u;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < vol; e += (long long)gridDim.x * blockDim.x) {
        const typename C2<R>::T a = acc[base + e], b = prev[base + e];
        const float am = hypotf((float)a.x, (float)a.y);
        const float dm = hypotf((float)(a.x - b.x), (float)(a.y - b.y)) * tf;
        amax = fmaxf(amax, am);
        if (dm > tol * fmaxf(am, floor_a)) viol = 1u;
        prev[base + e] = a;
    }
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmaxf(amax, __shfl_down_sync(0xffffffffu, amax, o));
        viol |= __shfl_down_sync(0xffffffffu, viol, o);
    }
    __shared__ float sa[8];
    __shared__ unsigned sv[8];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sa[wid] = amax; sv[wid] = viol; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { amax = fmaxf(amax, sa[k]); viol |= sv[k]; }
        atomicMax(stats + f, __float_as_uint(amax));          // non-negative floats order like their bits
        if (viol) atomicOr(stats + nf + f, 1u);
    }
}

template <typename R>
cudaError_t launch_es_vol_stats(const typename C2<R>::T *acc, typename C2<R>::T *prev, long long vol, int S, int nf,
                                double tol, double floor_frac, const EsTail &tail, unsigned *stats, cudaStream_t st) {
    const dim3 grid((unsigned)std::min<long long>((vol + 255) / 256, 64), (unsigned)(S * 3 * nf));
    k_es_vol_stats<R><<<grid, 256, 0, st>>>(acc, prev, vol, nf, (float)tol, (float)floor_frac, tail, stats);
    g_launches++;
    return cudaGetLastError();
}

__global__ void k_es_vol_decide(unsigned *stats, int nf, int chunk, int last, int steps_at, int *state) {
    if (state[0]) return;
    bool done = last != 0;
    if (!done && chunk >= 1) {
        done = true;
        for (int f = 0; f < nf; ++f)
            if (stats[nf + f]) done = false;
    }
    for (int f = 0; f < nf; ++f) stats[2 * nf + f] = stats[f];   // this check's maxima for the next one
    if (done) { state[1] = steps_at; state[0] = 1; }
}

cudaError_t launch_es_vol_decide(unsigned *stats, int nf, int chunk, int last, int steps_at, int *state,
                                 cudaStream_t st) {
    k_es_vol_decide<<<1, 1, 0, st>>>(stats, nf, chunk, last, steps_at, state);
    g_launches++;
    return cudaGetLastError();
}

template cudaError_t launch_es_vol_stats<float>(const float2 *, float2 *, long long, int, int, double, double,
                                                const EsTail &, unsigned *, cudaStream_t);
template cudaError_t launch_es_vol_stats<double>(const double2 *, double2 *, long long, int, int, double, double,
                                                 const EsTail &, unsigned *, cudaStream_t);

// ---------------------------------------------------------------------------
// misfit and weighted residual (Sec. 3.1, Eq. 7), one block
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_misfit(int n, const double *dobs, const double *dsyn, const double *w,
                                                 double *resid, double *phi) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const double wt = w ? w[t] : 1.0;
        const double rr = dobs[2 * t] - dsyn[2 * t], ri = dobs[2 * t + 1] - dsyn[2 * t + 1];
        acc += wt * wt * (rr * rr + ri * ri);
        resid[2 * t] = wt * wt * rr;
        resid[2 * t + 1] = wt * wt * ri;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *phi = 0.5 * acc;
    }
}

cudaError_t launch_misfit(int n, const double *d_obs, const double *d_syn, const double *w, double *resid,
                          double *phi, cudaStream_t st) {
    k_misfit<<<1, 1024, 0, st>>>(n, d_obs, d_syn, w, resid, phi);
    g_launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Adjoint-source basis (Sec. 3.3), FP64.  B (2 nf x nt) is never stored: each
// thread walks a contiguous range of n and advances exp((-1+i) a_k t_n) by the
// complex factor exp((-1+i) a_k dt) per sample (the start of each range is
// evaluated directly).  Rows 0..nf-1 are the real parts, nf..2nf-1 the
// imaginary parts.
// ---------------------------------------------------------------------------
constexpr int kBT = 512;

struct BasisArgs {
    double dt; int nt; int nf; double a[kMaxFreq];
};

__device__ __forceinline__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

// z_k(n0) = exp((-1+i) a_k (n0+1/2) dt), step factor q_k = exp((-1+i) a_k dt)
__device__ __forceinline__ void phasor_start(const BasisArgs &b, int f, int n0, double &zr, double &zi, double &qr,
                                             double &qi) {
    const double t = (n0 + 0.5) * b.dt;
    double sn, cs;
    sincos(b.a[f] * t, &sn, &cs);
    const double e = exp(-b.a[f] * t);
    zr = e * cs; zi = e * sn;
    sincos(b.a[f] * b.dt, &sn, &cs);
    const double eq = exp(-b.a[f] * b.dt);
    qr = eq * cs; qi = eq * sn;
}

// Gram matrix G = B B^T (2nf x 2nf), one block per (row, col) pair with row <= col.
__global__ void __launch_bounds__(kBT) k_basis_gram(BasisArgs b, double *G) {
    __shared__ double red[kBT / 32];
    const int m = 2 * b.nf;
    const int r = blockIdx.x, c = blockIdx.y;
    if (r > c) return;
    const int chunk = (b.nt + kBT - 1) / kBT;
    const int n0 = threadIdx.x * chunk, n1 = min(n0 + chunk, b.nt);
    double acc = 0.0;
    if (n0 < n1) {
        const int fr = r % b.nf, fc = c % b.nf;
        double zr, zi, qr, qi, wr, wi, pr, pi;
        phasor_start(b, fr, n0, zr, zi, qr, qi);
        phasor_start(b, fc, n0, wr, wi, pr, pi);
        for (int n = n0; n < n1; ++n) {
            const double br = (r < b.nf) ? zr : zi;
            const double bc = (c < b.nf) ? wr : wi;
            acc += br * bc;
            double t = zr * qr - zi * qi; zi = zr * qi + zi * qr; zr = t;
            t = wr * pr - wi * pi; wi = wr * pi + wi * pr; wr = t;
        }
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) { G[r * m + c] = acc; G[c * m + r] = acc; }
}

// gamma = gamma_rel * lambda_max(G) by power iteration (G is symmetric positive semi-definite).
__global__ void k_basis_gamma(const double *G, int m, double gamma, int rel, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (!rel) { out[0] = gamma; return; }
    double v[2 * kMaxFreq], w[2 * kMaxFreq];
    for (int i = 0; i < m; ++i) v[i] = 1.0 / (1.0 + i);
    double lam = 0.0;
    for (int it = 0; it < 500; ++it) {
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int j = 0; j < m; ++j) s += G[i * m + j] * v[j];
            w[i] = s;
            nrm += s * s;
        }
        nrm = sqrt(nrm);
        if (nrm == 0.0) break;
        for (int i = 0; i < m; ++i) v[i] = w[i] / nrm;
        lam = nrm;
    }
    out[0] = gamma * lam;
}

// CGNR on (B^T B + gamma I) x = B^T e_j, one block per column j (Sec. 3.3).
// x is written into basis[n*2nf + j]; P and Sv are [2nf][nt] scratch rows.
__global__ void __launch_bounds__(kBT) k_basis_cgnr(BasisArgs b, const double *gamma_p, int max_iter, double tol,
                                                   double *basis, double *scratch, int *iters) {
    __shared__ double red[kBT / 32];
    __shared__ double rvec[2 * kMaxFreq], qvec[2 * kMaxFreq];
    const int m = 2 * b.nf, col = blockIdx.x;
    const double gamma = gamma_p[0];
    double *P = scratch + (long long)col * 2 * b.nt;
    double *Sv = P + b.nt;
    const int chunk = (b.nt + kBT - 1) / kBT;
    const int n0 = threadIdx.x * chunk, n1 = min(n0 + chunk, b.nt);
    if (threadIdx.x < m) rvec[threadIdx.x] = (threadIdx.x == col) ? 1.0 : 0.0;
    __syncthreads();

    // s = B^T r - gamma x with x = 0, p = s
    double gl = 0.0;
    double zr[kMaxFreq], zi[kMaxFreq], qr[kMaxFreq], qi[kMaxFreq];
    if (n0 < n1) {
        for (int f = 0; f < b.nf; ++f) phasor_start(b, f, n0, zr[f], zi[f], qr[f], qi[f]);
        for (int n = n0; n < n1; ++n) {
            double s = 0.0;
            for (int f = 0; f < b.nf; ++f) {
                s += zr[f] * rvec[f] + zi[f] * rvec[b.nf + f];
                double t = zr[f] * qr[f] - zi[f] * qi[f]; zi[f] = zr[f] * qi[f] + zi[f] * qr[f]; zr[f] = t;
            }
            Sv[n] = s; P[n] = s;
            basis[(long long)n * m + col] = 0.0;
            gl += s * s;
        }
    }
    double gam = block_sum(gl, red);
    const double g0 = gam;
    int it = 0;
    for (; it < max_iter; ++it) {
        if (!(sqrt(gam) > tol * sqrt(g0))) break;
        // q = B p, pp = ||p||^2
        double ql[2 * kMaxFreq];
        for (int i = 0; i < m; ++i) ql[i] = 0.0;
        double pp = 0.0;
        if (n0 < n1) {
            for (int f = 0; f < b.nf; ++f) phasor_start(b, f, n0, zr[f], zi[f], qr[f], qi[f]);
            for (int n = n0; n < n1; ++n) {
                const double pn = P[n];
                pp += pn * pn;
                for (int f = 0; f < b.nf; ++f) {
                    ql[f] += zr[f] * pn;
                    ql[b.nf + f] += zi[f] * pn;
                    double t = zr[f] * qr[f] - zi[f] * qi[f]; zi[f] = zr[f] * qi[f] + zi[f] * qr[f]; zr[f] = t;
                }
            }
        }
        for (int i = 0; i < m; ++i) {
            const double v = block_sum(ql[i], red);
            if (threadIdx.x == 0) qvec[i] = v;
        }
        pp = block_sum(pp, red);
        __syncthreads();
        double qq = 0.0;
        for (int i = 0; i < m; ++i) qq += qvec[i] * qvec[i];
        const double alpha = gam / (qq + gamma * pp);
        __syncthreads();
        if (threadIdx.x < m) rvec[threadIdx.x] -= alpha * qvec[threadIdx.x];
        __syncthreads();
        // x += alpha p; s = B^T r - gamma x; ||s||^2
        gl = 0.0;
        if (n0 < n1) {
            for (int f = 0; f < b.nf; ++f) phasor_start(b, f, n0, zr[f], zi[f], qr[f], qi[f]);
            for (int n = n0; n < n1; ++n) {
                double x = basis[(long long)n * m + col] + alpha * P[n];
                basis[(long long)n * m + col] = x;
                double s = -gamma * x;
                for (int f = 0; f < b.nf; ++f) {
                    s += zr[f] * rvec[f] + zi[f] * rvec[b.nf + f];
                    double t = zr[f] * qr[f] - zi[f] * qi[f]; zi[f] = zr[f] * qi[f] + zi[f] * qr[f]; zr[f] = t;
                }
                Sv[n] = s;
                gl += s * s;
            }
        }
        const double gnew = block_sum(gl, red);
        const double beta = gnew / gam;
        gam = gnew;
        for (int n = n0; n < n1; ++n) P[n] = Sv[n] + beta * P[n];
        __syncthreads();
    }
    if (threadIdx.x == 0) iters[col] = it;
}

// fit: max_i |(B B+)_{i,col} - delta_{i,col}|, one block per column
__global__ void __launch_bounds__(kBT) k_basis_fit(BasisArgs b, const double *basis, double *fit) {
    __shared__ double red[kBT / 32];
    const int m = 2 * b.nf, col = blockIdx.x;
    const int chunk = (b.nt + kBT - 1) / kBT;
    const int n0 = threadIdx.x * chunk, n1 = min(n0 + chunk, b.nt);
    double ql[2 * kMaxFreq];
    for (int i = 0; i < m; ++i) ql[i] = 0.0;
    if (n0 < n1) {
        double zr[kMaxFreq], zi[kMaxFreq], qr[kMaxFreq], qi[kMaxFreq];
        for (int f = 0; f < b.nf; ++f) phasor_start(b, f, n0, zr[f], zi[f], qr[f], qi[f]);
        for (int n = n0; n < n1; ++n) {
            const double x = basis[(long long)n * m + col];
            for (int f = 0; f < b.nf; ++f) {
                ql[f] += zr[f] * x;
                ql[b.nf + f] += zi[f] * x;
                double t = zr[f] * qr[f] - zi[f] * qi[f]; zi[f] = zr[f] * qi[f] + zi[f] * qr[f]; zr[f] = t;
            }
        }
    }
    double worst = 0.0;
    for (int i = 0; i < m; ++i) {
        const double v = block_sum(ql[i], red);
        worst = fmax(worst, fabs(v - (i == col ? 1.0 : 0.0)));
    }
    if (threadIdx.x == 0) fit[col] = worst;
}

cudaError_t launch_basis(double dt, int nt, const double *a, int nf, double gamma, int gamma_rel, int max_iter,
                         double tol, double *basis, double *scratch, double *gram, double *out_scalars,
                         int *out_iters, cudaStream_t st) {
    BasisArgs b;
    b.dt = dt; b.nt = nt; b.nf = nf;
    for (int f = 0; f < kMaxFreq; ++f) b.a[f] = (f < nf) ? a[f] : 0.0;
    const int m = 2 * nf;
    k_basis_gram<<<dim3(m, m), kBT, 0, st>>>(b, gram);
    k_basis_gamma<<<1, 32, 0, st>>>(gram, m, gamma, gamma_rel, out_scalars);
    k_basis_cgnr<<<m, kBT, 0, st>>>(b, out_scalars, max_iter, tol, basis, scratch, out_iters);
    k_basis_fit<<<m, kBT, 0, st>>>(b, basis, out_scalars + 1);
    g_launches += 4;
    return cudaGetLastError();
}

// colmap[pos[u]] = val[u]: sets the column map of the injection taps
__global__ void k_scatter_int2(int2 *dst, const long long *pos, const int2 *val, int n) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u < n) dst[pos[u]] = val[u];
}

cudaError_t launch_scatter_int2(int2 *dst, const long long *pos, const int2 *val, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_scatter_int2<<<(n + 255) / 256, 256, 0, st>>>(dst, pos, val, n);
    g_launches++;
    return cudaGetLastError();
}

template cudaError_t launch_coef_init<float>(const GeoD &, const float *, const float *, float *, double, int *,
                                             cudaStream_t);
template cudaError_t launch_coef_init<double>(const GeoD &, const double *, const double *, double *, double, int *,
                                              cudaStream_t);
template cudaError_t launch_finalize_volume<float>(float2 *, const float2 *, long long, int, int, const double2 *,
                                                   cudaStream_t);
template cudaError_t launch_finalize_volume<double>(double2 *, const double2 *, long long, int, int,
                                                    const double2 *, cudaStream_t);
template cudaError_t launch_gradient<float>(const GeoD &, const float *, const float2 *, const float2 *, int, int,
                                            int, bool, float *, float *, cudaStream_t);
template cudaError_t launch_gradient<double>(const GeoD &, const double *, const double2 *, const double2 *, int,
                                             int, int, bool, double *, double *, cudaStream_t);
template cudaError_t launch_grad_cells<float>(const GeoD &, const float *, const float *, int, bool, float *,
                                              cudaStream_t);
template cudaError_t launch_grad_cells<double>(const GeoD &, const double *, const double *, int, bool, double *,
                                               cudaStream_t);

}  // namespace csem
