// Fourth-order staggered H and E steps on the non-uniform grid (Sec. 2,
// Eq. 4 with the high-order differences of the paper's engine; the weights are
// described in csem_ho.cuh).  One thread per (i, j) column and KZ planes, the
// four-point neighbours read through the read-only cache; the CPML memory is
// touched only inside its slabs.  E lives in the same ring of snapshots as in
// the second-order kernels (E^{n+1} is written to slot n+1 from slot n), and the
// E kernel applies the source injection of its column's taps.
#include "csem_ho.cuh"

namespace csem {

namespace {

constexpr int kHoX = 32, kHoY = 8, kHoZ = 4;

template <typename R> __device__ __forceinline__ R ld(const R *p) { return __ldg(p); }

// d/da at the half node pos (of n) of a node-located field F, F[at] at node pos
template <typename R>
__device__ __forceinline__ R d_half(const R *__restrict__ F, long long at, long long s, int pos, int n,
                                    const R *__restrict__ w) {
    const R *wr = w + 4 * pos;
    R d = ld(wr + 1) * ld(F + at) + ld(wr + 2) * ld(F + at + s);
    if (pos >= 1 && pos <= n - 2) d = ld(wr) * ld(F + at - s) + d + ld(wr + 3) * ld(F + at + 2 * s);
    return d;
}

// d/da at the node pos (of n) of a half-node-located field F, F[at] at half node pos
template <typename R>
__device__ __forceinline__ R d_node(const R *__restrict__ F, long long at, long long s, int pos, int n,
                                    const R *__restrict__ w) {
    const R *wr = w + 4 * pos;
    R d = ld(wr + 1) * ld(F + at - s) + ld(wr + 2) * ld(F + at);
    if (pos >= 2 && pos <= n - 2) d = ld(wr) * ld(F + at - 2 * s) + d + ld(wr + 3) * ld(F + at + s);
    return d;
}

// psi <- b psi + a d inside the slab, d + psi returned
template <typename R>
__device__ __forceinline__ R pml(R d, bool in, R b, R a, R *ps) {
    if (!in) return d;
    const R v = b * *ps + a * d;
    *ps = v;
    return d + v;
}

template <typename R>
__global__ void __launch_bounds__(kHoX *kHoY) k_h_ho(const StepParams<R> p, const HoTab<R> w, const int jstep) {
    const int i = blockIdx.x * kHoX + threadIdx.x;
    const int j = blockIdx.y * kHoY + threadIdx.y;
    const int nzb = (p.NZ + kHoZ - 1) / kHoZ;
    const int s = blockIdx.z / nzb, k0 = (blockIdx.z % nzb) * kHoZ;
    if (i >= p.NX || j >= p.NY) return;
    const int n = *p.step + jstep;
    const long long vol = p.vol, plane = p.plane, pitch = p.pitch;
    const R *__restrict__ Ex = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * vol;
    const R *__restrict__ Ey = Ex + vol;
    const R *__restrict__ Ez = Ex + 2 * vol;
    R *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    R *__restrict__ Hy = Hx + vol;
    R *__restrict__ Hz = Hx + 2 * vol;
    R *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml;
    const R cH = p.cH;
    const bool xin = slab_half(i, nx, npml) >= 0, yin = slab_half(j, ny, npml) >= 0;
    const R bx = xin ? ld(p.ax.b_h + i) : R(0), ax_ = xin ? ld(p.ax.a_h + i) : R(0);
    const R by = yin ? ld(p.ay.b_h + j) : R(0), ay_ = yin ? ld(p.ay.a_h + j) : R(0);
    for (int k = k0; k < k0 + kHoZ && k < p.NZ; ++k) {
        const long long idx = (long long)k * plane + (long long)j * pitch + i;
        const bool zin = slab_half(k, nz, npml) >= 0;
        const R bz = zin ? ld(p.az.b_h + k) : R(0), az_ = zin ? ld(p.az.a_h + k) : R(0);
        if (j < ny && k < nz) {            // Hx at (i, j+1/2, k+1/2)
            const R a = pml(d_half(Ez, idx, pitch, j, ny, w.wyh), yin, by, ay_, P + idx);
            const R b = pml(d_half(Ey, idx, plane, k, nz, w.wzh), zin, bz, az_, P + vol + idx);
            Hx[idx] -= cH * (a - b);
        }
        if (i < nx && k < nz) {            // Hy at (i+1/2, j, k+1/2)
            const R a = pml(d_half(Ex, idx, plane, k, nz, w.wzh), zin, bz, az_, P + 2 * vol + idx);
            const R b = pml(d_half(Ez, idx, 1LL, i, nx, w.wxh), xin, bx, ax_, P + 3 * vol + idx);
            Hy[idx] -= cH * (a - b);
        }
        if (i < nx && j < ny) {            // Hz at (i+1/2, j+1/2, k)
            const R a = pml(d_half(Ey, idx, 1LL, i, nx, w.wxh), xin, bx, ax_, P + 4 * vol + idx);
            const R b = pml(d_half(Ex, idx, pitch, j, ny, w.wyh), yin, by, ay_, P + 5 * vol + idx);
            Hz[idx] -= cH * (a - b);
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kHoX *kHoY) k_e_ho(const StepParams<R> p, const HoTab<R> w, const int jstep) {
    const int i = blockIdx.x * kHoX + threadIdx.x;
    const int j = blockIdx.y * kHoY + threadIdx.y;
    const int nzb = (p.NZ + kHoZ - 1) / kHoZ;
    const int s = blockIdx.z / nzb, k0 = (blockIdx.z % nzb) * kHoZ;
    if (i >= p.NX || j >= p.NY) return;
    const int n = *p.step + jstep;
    const long long vol = p.vol, plane = p.plane, pitch = p.pitch;
    const R *__restrict__ Eo = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * vol;
    R *__restrict__ En = p.ering + (long long)s * p.ering_stride + (long long)((n + 1) % p.nslot) * 3 * vol;
    const R *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    const R *__restrict__ Hy = Hx + vol;
    const R *__restrict__ Hz = Hx + 2 * vol;
    R *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml;
    const bool xin = slab_node(i, nx, npml) >= 0, yin = slab_node(j, ny, npml) >= 0;
    const R bx = xin ? ld(p.ax.b_n + i) : R(0), ax_ = xin ? ld(p.ax.a_n + i) : R(0);
    const R by = yin ? ld(p.ay.b_n + j) : R(0), ay_ = yin ? ld(p.ay.a_n + j) : R(0);
    const bool ix = (i >= 1 && i < nx), jy = (j >= 1 && j < ny);
    for (int k = k0; k < k0 + kHoZ && k < p.NZ; ++k) {
        const long long idx = (long long)k * plane + (long long)j * pitch + i;
        const bool zin = slab_node(k, nz, npml) >= 0;
        const R bz = zin ? ld(p.az.b_n + k) : R(0), az_ = zin ? ld(p.az.a_n + k) : R(0);
        const bool kz = (k >= 1 && k < nz);
        if (i < nx && jy && kz) {          // Ex at (i+1/2, j, k)
            const R a = pml(d_node(Hz, idx, pitch, j, ny, w.wyn), yin, by, ay_, P + 6 * vol + idx);
            const R b = pml(d_node(Hy, idx, plane, k, nz, w.wzn), zin, bz, az_, P + 7 * vol + idx);
            En[idx] = ld(Eo + idx) + ld(p.cE + idx) * (a - b);
        }
        if (j < ny && ix && kz) {          // Ey at (i, j+1/2, k)
            const R a = pml(d_node(Hx, idx, plane, k, nz, w.wzn), zin, bz, az_, P + 8 * vol + idx);
            const R b = pml(d_node(Hz, idx, 1LL, i, nx, w.wxn), xin, bx, ax_, P + 9 * vol + idx);
            En[vol + idx] = ld(Eo + vol + idx) + ld(p.cE + vol + idx) * (a - b);
        }
        if (k < nz && ix && jy) {          // Ez at (i, j, k+1/2)
            const R a = pml(d_node(Hy, idx, 1LL, i, nx, w.wxn), xin, bx, ax_, P + 10 * vol + idx);
            const R b = pml(d_node(Hx, idx, pitch, j, ny, w.wyn), yin, by, ay_, P + 11 * vol + idx);
            En[2 * vol + idx] = ld(Eo + 2 * vol + idx) + ld(p.cE + 2 * vol + idx) * (a - b);
        }
    }
    // source term E^{n+1} -= dt/eps J'^{n+1/2} for the taps of this column and planes
    if (p.colmap) {
        const int2 cm = p.colmap[s * p.colmap_stride + (long long)j * pitch + i];
        for (int u = cm.x; u < cm.x + cm.y; ++u) {
            const Tap tp = p.itaps[(long long)s * p.itap_stride + u];
            const int k = (int)(tp.idx / plane);
            if (k < k0 || k >= k0 + kHoZ) continue;
            const double *cf = p.coef + ((long long)s * p.n_emit + tp.emit) * p.J;
            const double *T = p.T + (long long)n * p.J;
            double amp = 0.0;
            for (int jj = 0; jj < p.J; ++jj) amp += cf[jj] * T[jj];
            const long long o = (long long)tp.comp * vol + tp.idx;
            const double add = -(double)p.cE[o] * tp.w * amp;
            if (add != 0.0) En[o] += (R)add;
        }
    }
}

}  // namespace

template <typename R>
cudaError_t launch_ho(const StepParams<R> &p, const HoTab<R> &w, int S, int jstep, cudaStream_t st, int which) {
    const dim3 blk(kHoX, kHoY);
    const dim3 grid((p.NX + kHoX - 1) / kHoX, (p.NY + kHoY - 1) / kHoY, S * ((p.NZ + kHoZ - 1) / kHoZ));
    if (which & 1) {
        k_h_ho<R><<<grid, blk, 0, st>>>(p, w, jstep);
        g_launches++;
    }
    if (which & 4) {
        k_e_ho<R><<<grid, blk, 0, st>>>(p, w, jstep);
        g_launches++;
    }
    return cudaGetLastError();
}

template cudaError_t launch_ho<float>(const StepParams<float> &, const HoTab<float> &, int, int, cudaStream_t, int);
template cudaError_t launch_ho<double>(const StepParams<double> &, const HoTab<double> &, int, int, cudaStream_t,
                                       int);

}  // namespace csem
