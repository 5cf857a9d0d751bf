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

// ---------------------------------------------------------------------------
// Lean FP32 fourth-order kernels: two consecutive cells (i, i+1) of one (j, k) row
// per thread (8-byte accesses), 32 x 4-thread blocks with a register budget, KZ
// planes per thread marched along z with the four planes of the z derivatives in
// a register window (one new plane loaded per step), the x and y neighbours of a
// plane loaded together, and no branches on the boundary rows: their two-point
// weights have zero outer entries and the neighbours they would read outside the
// lattice are clamped to the cell itself.  E is advanced with dt/eps zeroed on the
// PEC edges, so every component is written unconditionally.  The CPML memory
// (12 field-layout arrays per source) is touched only in its slabs; the source
// taps come from the per-chunk increments.  The work domain is the cell range
// [0,nx) x [0,ny) x [0,nz) (H outside it never changes).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 f2g(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float2 f2w(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void f2s(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ float4 f4g(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
// w . (a, b, c, d) for both cells of the pair
__device__ __forceinline__ float2 dot4(const float4 &w, float2 a, float2 b, float2 c, float2 d) {
    return make_float2(w.x * a.x + w.y * b.x + w.z * c.x + w.w * d.x, w.x * a.y + w.y * b.y + w.z * c.y + w.w * d.y);
}
// x derivative of the pair from five consecutive values f0 .. f4 (cell i uses f0..f3, cell i+1 f1..f4)
__device__ __forceinline__ float2 dx5(const float4 &w0, const float4 &w1, float f0, float f1, float f2, float f3,
                                      float f4) {
    return make_float2(w0.x * f0 + w0.y * f1 + w0.z * f2 + w0.w * f3, w1.x * f1 + w1.y * f2 + w1.z * f3 + w1.w * f4);
}
__device__ __forceinline__ void pml2(float2 &d, bool in, float b, float a, float *ps) {
    if (!in) return;
    float2 v = f2w(ps);
    v.x = b * v.x + a * d.x; v.y = b * v.y + a * d.y;
    f2s(ps, v);
    d.x += v.x; d.y += v.y;
}
__device__ __forceinline__ void pml2x(float2 &d, bool in0, bool in1, float2 b, float2 a, float *ps) {
    if (!in0 && !in1) return;
    float2 v = f2w(ps);
    v.x = b.x * v.x + a.x * d.x; v.y = b.y * v.y + a.y * d.y;
    f2s(ps, v);
    d.x += v.x; d.y += v.y;
}
__device__ __forceinline__ float3 ho_taps(const int *__restrict__ tk, const float *__restrict__ inc, int k, int2 cm) {
    float3 r = make_float3(0.f, 0.f, 0.f);
    for (int u = cm.x; u < cm.x + cm.y; ++u) {
        const int code = __ldg(tk + u);
        const float v = __ldg(inc + u);
        if ((code >> 2) != k) continue;
        if ((code & 3) == 0) r.x += v;
        else if ((code & 3) == 1) r.y += v;
        else r.z += v;
    }
    return r;
}

template <int KZ, int MINB>
__global__ void __launch_bounds__(128, MINB) k_h_ho4(const StepParams<float> p, const HoTab<float> w, const int jstep) {
    const int i = (blockIdx.x * 32 + threadIdx.x) * 2;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int nkb = (p.nz + KZ - 1) / KZ;
    const int S = gridDim.z / nkb;
    const int s = blockIdx.z % S, k0 = (blockIdx.z / S) * KZ;
    if (i >= p.nx || j >= p.ny) return;
    const int k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;
    const float *__restrict__ Ex = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    const float *__restrict__ Ey = Ex + vol;
    const float *__restrict__ Ez = Ex + 2 * vol;
    float *__restrict__ H = p.H + (long long)s * 3 * vol;
    float *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    const float cH = p.cH;
    // neighbours, clamped on the lattice: column i-1; rows j-1, j+2 (column i+3 lies in the
    // lattice row or its padding, and only the last half node's zero weight meets it there)
    const int im = (i > 0) ? -1 : 0;
    const int jm = (j > 0) ? -pitch : 0, jp2 = (j + 2 <= ny) ? 2 * pitch : (ny - j) * pitch;
    const float4 wx0 = f4g(w.wxh + 4 * i), wx1 = f4g(w.wxh + 4 * (i + 1)), wy = f4g(w.wyh + 4 * j);
    const bool xs0 = slab_half(i, nx, npml) >= 0, xs1 = slab_half(i + 1, nx, npml) >= 0;
    const bool ys = slab_half(j, ny, npml) >= 0;
    const float2 bx = make_float2(__ldg(p.lx.b_h + i), __ldg(p.lx.b_h + i + 1));
    const float2 ax = make_float2(__ldg(p.lx.a_h + i), __ldg(p.lx.a_h + i + 1));
    const float by = __ldg(p.ly.b_h + j), ay = __ldg(p.ly.a_h + j);
    // z window of Ex, Ey at the thread's cells: planes k-1, k, k+1 (k+2 loaded per step)
    const int base = j * pitch + i;
    int km = (k0 > 0) ? k0 - 1 : 0;
    float2 xa = f2g(Ex + km * plane + base), xb = f2g(Ex + k0 * plane + base), xc = f2g(Ex + (k0 + 1) * plane + base);
    float2 ya = f2g(Ey + km * plane + base), yb = f2g(Ey + k0 * plane + base), yc = f2g(Ey + (k0 + 1) * plane + base);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk) {
        const int k = k0 + kk;
        if (k >= k1) break;
        const int idx = k * plane + base;
        const int kp2 = (k + 2 <= nz) ? k + 2 : nz;
        const float2 xd = f2g(Ex + kp2 * plane + base), yd = f2g(Ey + kp2 * plane + base);
        const float4 wz = f4g(w.wzh + 4 * k);
        // x neighbours of Ey, Ez (plane k): values at i-1 .. i+3
        const float eym = __ldg(Ey + idx + im), ezm = __ldg(Ez + idx + im);
        const float2 ez01 = f2g(Ez + idx), ey23 = f2g(Ey + idx + 2), ez23 = f2g(Ez + idx + 2);
        // y neighbours of Ex, Ez (plane k): rows j-1, j+1, j+2
        const float2 exm = f2g(Ex + idx + jm), exp1 = f2g(Ex + idx + pitch), exp2 = f2g(Ex + idx + jp2);
        const float2 ezm2 = f2g(Ez + idx + jm), ezp1 = f2g(Ez + idx + pitch), ezp2 = f2g(Ez + idx + jp2);
        float2 hx = f2w(H + idx), hy = f2w(H + vol + idx), hz = f2w(H + 2 * vol + idx);
        float2 dEz_dy = dot4(wy, ezm2, ez01, ezp1, ezp2), dEy_dz = dot4(wz, ya, yb, yc, yd);
        float2 dEx_dz = dot4(wz, xa, xb, xc, xd), dEz_dx = dx5(wx0, wx1, ezm, ez01.x, ez01.y, ez23.x, ez23.y);
        float2 dEy_dx = dx5(wx0, wx1, eym, yb.x, yb.y, ey23.x, ey23.y), dEx_dy = dot4(wy, exm, xb, exp1, exp2);
        const bool zs = slab_half(k, nz, npml) >= 0;
        if (ys || zs || xs0 || xs1) {
            const float bz = __ldg(p.lz.b_h + k), az = __ldg(p.lz.a_h + k);
            pml2(dEz_dy, ys, by, ay, P + idx);
            pml2(dEy_dz, zs, bz, az, P + vol + idx);
            pml2(dEx_dz, zs, bz, az, P + 2 * vol + idx);
            pml2x(dEz_dx, xs0, xs1, bx, ax, P + 3 * vol + idx);
            pml2x(dEy_dx, xs0, xs1, bx, ax, P + 4 * vol + idx);
            pml2(dEx_dy, ys, by, ay, P + 5 * vol + idx);
        }
        hx.x -= cH * (dEz_dy.x - dEy_dz.x); hx.y -= cH * (dEz_dy.y - dEy_dz.y);
        hy.x -= cH * (dEx_dz.x - dEz_dx.x); hy.y -= cH * (dEx_dz.y - dEz_dx.y);
        hz.x -= cH * (dEy_dx.x - dEx_dy.x); hz.y -= cH * (dEy_dx.y - dEx_dy.y);
        f2s(H + idx, hx);
        f2s(H + vol + idx, hy);
        f2s(H + 2 * vol + idx, hz);
        xa = xb; xb = xc; xc = xd;
        ya = yb; yb = yc; yc = yd;
    }
}

template <int KZ, int MINB>
__global__ void __launch_bounds__(128, MINB) k_e_ho4(const StepParams<float> p, const HoTab<float> w, const int jstep) {
    const int i = (blockIdx.x * 32 + threadIdx.x) * 2;
    const int j = blockIdx.y * 4 + threadIdx.y;
    const int nkb = (p.nz + KZ - 1) / KZ;
    const int S = gridDim.z / nkb;
    const int s = blockIdx.z % S, k0 = (blockIdx.z / S) * KZ;
    if (i >= p.nx || j >= p.ny) return;
    const int k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;
    const float *__restrict__ ring = p.ering + (long long)s * p.ering_stride;
    const float *__restrict__ Eo = ring + (long long)(n % p.nslot) * 3 * p.vol;
    float *__restrict__ En = const_cast<float *>(ring) + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    const float *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    const float *__restrict__ Hy = Hx + vol;
    const float *__restrict__ Hz = Hx + 2 * vol;
    float *__restrict__ P = p.psi + (long long)s * p.psi_stride + 6LL * vol;
    const float *__restrict__ cE = p.cEm;
    // neighbours, clamped on the lattice: columns i-2; rows j-2, j-1
    const int im2 = (i >= 2) ? -2 : -i;
    const int jm2 = (j >= 2) ? -2 * pitch : -j * pitch, jm1 = (j >= 1) ? -pitch : 0;
    const float4 wx0 = f4g(w.wxn + 4 * i), wx1 = f4g(w.wxn + 4 * (i + 1)), wy = f4g(w.wyn + 4 * j);
    const bool xs0 = slab_node(i, nx, npml) >= 0, xs1 = slab_node(i + 1, nx, npml) >= 0;
    const bool ys = slab_node(j, ny, npml) >= 0;
    const float2 bx = make_float2(__ldg(p.lx.b_n + i), __ldg(p.lx.b_n + i + 1));
    const float2 ax = make_float2(__ldg(p.lx.a_n + i), __ldg(p.lx.a_n + i + 1));
    const float by = __ldg(p.ly.b_n + j), ay = __ldg(p.ly.a_n + j);
    const bool taps = p.colmap && p.inc && p.tflag[s * p.tflag_stride + j * p.nseg + (i >> 5)];
    // z window of Hx, Hy at the thread's cells: planes k-2, k-1, k (k+1 loaded per step)
    const int base = j * pitch + i;
    const int ka = (k0 >= 2) ? k0 - 2 : 0, kb = (k0 >= 1) ? k0 - 1 : 0;
    float2 xa = f2g(Hx + ka * plane + base), xb = f2g(Hx + kb * plane + base), xc = f2g(Hx + k0 * plane + base);
    float2 ya = f2g(Hy + ka * plane + base), yb = f2g(Hy + kb * plane + base), yc = f2g(Hy + k0 * plane + base);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk) {
        const int k = k0 + kk;
        if (k >= k1) break;
        const int idx = k * plane + base;
        const float2 xd = f2g(Hx + idx + plane), yd = f2g(Hy + idx + plane);   // plane k+1 <= nz
        const float4 wz = f4g(w.wzn + 4 * k);
        // x neighbours of Hy, Hz (plane k): values at i-2 .. i+2
        const float2 hym = f2g(Hy + idx + im2), hzm = f2g(Hz + idx + im2);
        const float2 hz01 = f2g(Hz + idx);
        const float hy2 = __ldg(Hy + idx + 2), hz2 = __ldg(Hz + idx + 2);
        // y neighbours of Hx, Hz (plane k): rows j-2, j-1, j+1
        const float2 hxm2 = f2g(Hx + idx + jm2), hxm1 = f2g(Hx + idx + jm1), hxp1 = f2g(Hx + idx + pitch);
        const float2 hzm2 = f2g(Hz + idx + jm2), hzm1 = f2g(Hz + idx + jm1), hzp1 = f2g(Hz + idx + pitch);
        const float2 e0 = f2g(Eo + idx), e1 = f2g(Eo + vol + idx), e2 = f2g(Eo + 2 * vol + idx);
        const float2 c0 = f2g(cE + idx), c1 = f2g(cE + vol + idx), c2 = f2g(cE + 2 * vol + idx);
        float2 dHz_dy = dot4(wy, hzm2, hzm1, hz01, hzp1), dHy_dz = dot4(wz, ya, yb, yc, yd);
        float2 dHx_dz = dot4(wz, xa, xb, xc, xd);
        float2 dHz_dx = dx5(wx0, wx1, hzm.x, hzm.y, hz01.x, hz01.y, hz2);
        float2 dHy_dx = dx5(wx0, wx1, hym.x, hym.y, yc.x, yc.y, hy2);
        float2 dHx_dy = dot4(wy, hxm2, hxm1, xc, hxp1);
        const bool zs = slab_node(k, nz, npml) >= 0;
        if (ys || zs || xs0 || xs1) {
            const float bz = __ldg(p.lz.b_n + k), az = __ldg(p.lz.a_n + k);
            pml2(dHz_dy, ys, by, ay, P + idx);
            pml2(dHy_dz, zs, bz, az, P + vol + idx);
            pml2(dHx_dz, zs, bz, az, P + 2 * vol + idx);
            pml2x(dHz_dx, xs0, xs1, bx, ax, P + 3 * vol + idx);
            pml2x(dHy_dx, xs0, xs1, bx, ax, P + 4 * vol + idx);
            pml2(dHx_dy, ys, by, ay, P + 5 * vol + idx);
        }
        float2 ex = make_float2(e0.x + c0.x * (dHz_dy.x - dHy_dz.x), e0.y + c0.y * (dHz_dy.y - dHy_dz.y));
        float2 ey = make_float2(e1.x + c1.x * (dHx_dz.x - dHz_dx.x), e1.y + c1.y * (dHx_dz.y - dHz_dx.y));
        float2 ez = make_float2(e2.x + c2.x * (dHy_dx.x - dHx_dy.x), e2.y + c2.y * (dHy_dx.y - dHx_dy.y));
        if (taps) {
            const int2 *cm = p.colmap + (long long)s * p.colmap_stride + j * pitch + i;
            const int *tk = p.tapk + (long long)s * p.itap_stride;
            const float *inc = p.inc + ((long long)jstep * S + s) * p.inc_ntl;
            const int2 cc0 = __ldg(cm), cc1 = __ldg(cm + 1);
            if (cc0.y) { const float3 a = ho_taps(tk, inc, k, cc0); ex.x += a.x; ey.x += a.y; ez.x += a.z; }
            if (cc1.y) { const float3 a = ho_taps(tk, inc, k, cc1); ex.y += a.x; ey.y += a.y; ez.y += a.z; }
        }
        f2s(En + idx, ex);
        f2s(En + vol + idx, ey);
        f2s(En + 2 * vol + idx, ez);
        xa = xb; xb = xc; xc = xd;
        ya = yb; yb = yc; yc = yd;
    }
}

template <int KZ, int MB>
void go_ho4k(const StepParams<float> &p, const HoTab<float> &w, int S, int jstep, cudaStream_t st, bool h) {
    const dim3 grid((unsigned)((p.nx / 2 + 31) / 32), (unsigned)((p.ny + 3) / 4), (unsigned)(((p.nz + KZ - 1) / KZ) * S));
    if (h) k_h_ho4<KZ, MB><<<grid, dim3(32, 4), 0, st>>>(p, w, jstep);
    else k_e_ho4<KZ, MB><<<grid, dim3(32, 4), 0, st>>>(p, w, jstep);
}
template <int MB>
void go_ho4(const StepParams<float> &p, const HoTab<float> &w, int S, int jstep, cudaStream_t st, bool h, int kz) {
    if (kz == 2) go_ho4k<2, MB>(p, w, S, jstep, st, h);
    else if (kz == 4) go_ho4k<4, MB>(p, w, S, jstep, st, h);
    else go_ho4k<8, MB>(p, w, S, jstep, st, h);
}

}  // namespace

bool ho4_supported(int kz, int mb) { return (kz == 2 || kz == 4 || kz == 8) && (mb == 4 || mb == 6 || mb == 8); }

cudaError_t launch_ho4(const StepParams<float> &p, const HoTab<float> &w, int S, int jstep, cudaStream_t st, bool h,
                       int kz, int mb) {
    if (p.nx % 2 != 0 || !p.cEm || !p.lx.b_h || !ho4_supported(kz, mb)) return cudaErrorInvalidValue;
    if (mb == 4) go_ho4<4>(p, w, S, jstep, st, h, kz);
    else if (mb == 6) go_ho4<6>(p, w, S, jstep, st, h, kz);
    else go_ho4<8>(p, w, S, jstep, st, h, kz);
    g_launches++;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_ho(const StepParams<R> &p, const HoTab<R> &w, int S, int jstep, cudaStream_t st, int which) {
    bool lean_h = false, lean_e = false;       // FP32: the lean kernels for the halves that select them
    if constexpr (sizeof(R) == 4) {
        lean_h = p.LEAN_h != 0;
        lean_e = p.LEAN_e != 0;
    }
    const dim3 blk(kHoX, kHoY);
    const dim3 grid((p.NX + kHoX - 1) / kHoX, (p.NY + kHoY - 1) / kHoY, S * ((p.NZ + kHoZ - 1) / kHoZ));
    cudaError_t e = cudaSuccess;
    if (which & 1) {                           // the H half first, then the E half
        if (lean_h) {
            if constexpr (sizeof(R) == 4) e = launch_ho4(p, w, S, jstep, st, true, p.KZ_h, p.MB_h);
        } else {
            k_h_ho<R><<<grid, blk, 0, st>>>(p, w, jstep);
            g_launches++;
        }
    }
    if (e == cudaSuccess && (which & 4)) {
        if (lean_e) {
            if constexpr (sizeof(R) == 4) e = launch_ho4(p, w, S, jstep, st, false, p.KZ_e, p.MB_e);
        } else {
            k_e_ho<R><<<grid, blk, 0, st>>>(p, w, jstep);
            g_launches++;
        }
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template cudaError_t launch_ho<float>(const StepParams<float> &, const HoTab<float> &, int, int, cudaStream_t, int);
template cudaError_t launch_ho<double>(const StepParams<double> &, const HoTab<double> &, int, int, cudaStream_t,
                                       int);

}  // namespace csem
