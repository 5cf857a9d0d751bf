// FP32 H and E step kernels vectorised along x: each thread updates four
// consecutive cells (i .. i+3, i a multiple of 4) of one (j, k) row with 16-byte
// loads and stores, marching KZ planes along z.  The x-neighbour one cell up
// (for the H curl) or down (for the E curl) comes from the thread's own vector
// plus one scalar load.  The work domain is the cell range [0,nx) x [0,ny) x
// [0,nz): H faces and E edges outside it never change (tangential E is zero on
// the outer faces, so the normal H there keeps its initial zero).  Entries of a
// vector that are not on a component's updated lattice keep their old value.
// Same arithmetic, per entry, as the scalar kernels.
#include "csem_internal.cuh"

namespace csem {

namespace {

__device__ __forceinline__ float4 ld4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ldw4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float &at(float4 &v, int e) { return reinterpret_cast<float *>(&v)[e]; }
__device__ __forceinline__ float get(const float4 &v, int e) { return reinterpret_cast<const float *>(&v)[e]; }
__device__ __forceinline__ float4 sub(float4 a, float4 b) { return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
__device__ __forceinline__ float4 mul(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float4 mul(float4 a, float4 b) { return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w); }

// psi <- b psi + a d ;  d += psi   (four entries sharing b, a)
__device__ __forceinline__ void cpml4(float *ps, float b, float a, float4 &d) {
    float4 v = ldw4(ps);
    v.x = b * v.x + a * d.x; v.y = b * v.y + a * d.y; v.z = b * v.z + a * d.z; v.w = b * v.w + a * d.w;
    st4(ps, v);
    d.x += v.x; d.y += v.y; d.z += v.z; d.w += v.w;
}

}  // namespace

template <int KZ, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_h4(const StepParams<float> p, const int jstep) {
    const int qrow = p.pitch >> 2;
    const int t = blockIdx.x * kBlock + threadIdx.x;
    const int j = t / qrow;
    const int i = (t - j * qrow) << 2;
    if (j >= p.ny || i >= p.nx) return;
    const int s = blockIdx.z;
    const int n = *p.step + jstep;
    const int k0 = blockIdx.y * KZ;
    const int k1 = min(k0 + KZ, p.nz);
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;
    const float *__restrict__ E = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    const float *__restrict__ Ex = E;
    const float *__restrict__ Ey = E + vol;
    const float *__restrict__ Ez = E + 2 * vol;
    float *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    float *__restrict__ Hy = Hx + vol;
    float *__restrict__ Hz = Hx + 2 * vol;
    float *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    float *__restrict__ psx = P;
    float *__restrict__ psy = P + 6 * p.sx;
    float *__restrict__ psz = P + 6 * p.sx + 6 * p.sy;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml, np2 = 2 * npml;

    float4 ihx4;
#pragma unroll
    for (int e = 0; e < 4; ++e) at(ihx4, e) = (i + e < nx) ? __ldg(p.ax.ih_h + i + e) : 0.f;
    const bool xslab = (i < npml) || (i + 3 >= nx - npml);
    const float ihy = __ldg(p.ay.ih_h + j);
    const int syh = slab_half(j, ny, npml);
    float by = 0.f, ay = 0.f;
    if (syh >= 0) { by = __ldg(p.ay.b_h + j); ay = __ldg(p.ay.a_h + j); }
    const float cH = p.cH;
    const bool has4 = (i + 4 < pitch);

    int idx = k0 * plane + j * pitch + i;
    float4 exc = ld4(Ex + idx), eyc = ld4(Ey + idx);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= k1) break;
        const float4 ezc = ld4(Ez + idx);
        const float4 exk = ld4(Ex + idx + plane), eyk = ld4(Ey + idx + plane);
        const float4 ezj = ld4(Ez + idx + pitch), exj = ld4(Ex + idx + pitch);
        const float ez4 = has4 ? __ldg(Ez + idx + 4) : 0.f, ey4 = has4 ? __ldg(Ey + idx + 4) : 0.f;
        const float4 ezx = make_float4(ezc.y, ezc.z, ezc.w, ez4);
        const float4 eyx = make_float4(eyc.y, eyc.z, eyc.w, ey4);
        const float ihz = __ldg(p.az.ih_h + k);
        const int szh = slab_half(k, nz, npml);
        float bz = 0.f, az = 0.f;
        if (szh >= 0) { bz = __ldg(p.az.b_h + k); az = __ldg(p.az.a_h + k); }

        float4 dEz_dy = mul(sub(ezj, ezc), ihy), dEy_dz = mul(sub(eyk, eyc), ihz);   // Hx
        float4 dEx_dz = mul(sub(exk, exc), ihz), dEz_dx = mul(sub(ezx, ezc), ihx4);  // Hy
        float4 dEy_dx = mul(sub(eyx, eyc), ihx4), dEx_dy = mul(sub(exj, exc), ihy);  // Hz
        if (syh >= 0) {
            const int o = (k * np2 + syh) * pitch + i;
            cpml4(psy + o, by, ay, dEz_dy);
            cpml4(psy + p.sy + o, by, ay, dEx_dy);
        }
        if (szh >= 0) {
            const int o = (szh * p.NY + j) * pitch + i;
            cpml4(psz + o, bz, az, dEy_dz);
            cpml4(psz + p.sz + o, bz, az, dEx_dz);
        }
        if (xslab) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int ix = (i + e < nx) ? slab_half(i + e, nx, npml) : -1;
                if (ix < 0) continue;
                const float b = __ldg(p.ax.b_h + i + e), a = __ldg(p.ax.a_h + i + e);
                const int o = (k * p.NY + j) * np2 + ix;
                float &p0 = psx[o];
                p0 = b * p0 + a * get(dEz_dx, e);
                at(dEz_dx, e) += p0;
                float &p1 = psx[p.sx + o];
                p1 = b * p1 + a * get(dEy_dx, e);
                at(dEy_dx, e) += p1;
            }
        }
        float4 h = ldw4(Hx + idx);
        h.x -= cH * (dEz_dy.x - dEy_dz.x); h.y -= cH * (dEz_dy.y - dEy_dz.y);
        h.z -= cH * (dEz_dy.z - dEy_dz.z); h.w -= cH * (dEz_dy.w - dEy_dz.w);
        st4(Hx + idx, h);
        h = ldw4(Hy + idx);
        h.x -= cH * (dEx_dz.x - dEz_dx.x); h.y -= cH * (dEx_dz.y - dEz_dx.y);
        h.z -= cH * (dEx_dz.z - dEz_dx.z); h.w -= cH * (dEx_dz.w - dEz_dx.w);
        st4(Hy + idx, h);
        h = ldw4(Hz + idx);
        h.x -= cH * (dEy_dx.x - dEx_dy.x); h.y -= cH * (dEy_dx.y - dEx_dy.y);
        h.z -= cH * (dEy_dx.z - dEx_dy.z); h.w -= cH * (dEy_dx.w - dEx_dy.w);
        st4(Hz + idx, h);
        exc = exk;
        eyc = eyk;
    }
}

template <int KZ, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_e4(const StepParams<float> p, const int jstep) {
    const int qrow = p.pitch >> 2;
    const int t = blockIdx.x * kBlock + threadIdx.x;
    const int j = t / qrow;
    const int i = (t - j * qrow) << 2;
    if (j >= p.ny || i >= p.nx) return;
    const int s = blockIdx.z;
    const int n = *p.step + jstep;
    const int k0 = blockIdx.y * KZ;
    const int k1 = min(k0 + KZ, p.nz);
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;
    const float *__restrict__ Eo = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    float *__restrict__ En = p.ering + (long long)s * p.ering_stride + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    const float *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    const float *__restrict__ Hy = Hx + vol;
    const float *__restrict__ Hz = Hx + 2 * vol;
    const float *__restrict__ cE = p.cE;
    float *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    float *__restrict__ psx = P;
    float *__restrict__ psy = P + 6 * p.sx;
    float *__restrict__ psz = P + 6 * p.sx + 6 * p.sy;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml, np2 = 2 * npml;

    float4 ihx4;
    bool vx[4], vyz[4];    // Ex on lattice (i < nx); Ey / Ez off the x faces (1 <= i < nx)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        at(ihx4, e) = (i + e <= nx) ? __ldg(p.ax.ih_n + i + e) : 0.f;
        vx[e] = (i + e < nx);
        vyz[e] = (i + e >= 1) && (i + e < nx);
    }
    const bool xslab = (i < npml) || (i + 3 > nx - npml);
    const float ihy = __ldg(p.ay.ih_n + j);
    const int syn = slab_node(j, ny, npml);
    float by = 0.f, ay = 0.f;
    if (syn >= 0) { by = __ldg(p.ay.b_n + j); ay = __ldg(p.ay.a_n + j); }
    const bool jin = (j >= 1);

    int idx = k0 * plane + j * pitch + i;
    float4 hxm = (k0 > 0) ? ld4(Hx + idx - plane) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 hym = (k0 > 0) ? ld4(Hy + idx - plane) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= k1) break;
        const float4 hxc = ld4(Hx + idx), hyc = ld4(Hy + idx), hzc = ld4(Hz + idx);
        const float4 hzj = jin ? ld4(Hz + idx - pitch) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hxj = jin ? ld4(Hx + idx - pitch) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float hz1 = (i >= 1) ? __ldg(Hz + idx - 1) : 0.f, hy1 = (i >= 1) ? __ldg(Hy + idx - 1) : 0.f;
        const float4 hzx = make_float4(hz1, hzc.x, hzc.y, hzc.z);   // Hz at i-1 .. i+2
        const float4 hyx = make_float4(hy1, hyc.x, hyc.y, hyc.z);
        const float ihz = __ldg(p.az.ih_n + k);
        const int szn = slab_node(k, nz, npml);
        float bz = 0.f, az = 0.f;
        if (szn >= 0) { bz = __ldg(p.az.b_n + k); az = __ldg(p.az.a_n + k); }
        const bool kin = (k >= 1);

        float4 eo = ld4(Eo + idx);
        if (jin && kin) {                                         // Ex at (i+1/2, j, k)
            float4 dHz_dy = mul(sub(hzc, hzj), ihy), dHy_dz = mul(sub(hyc, hym), ihz);
            if (syn >= 0) cpml4(psy + 2 * p.sy + (k * np2 + syn) * pitch + i, by, ay, dHz_dy);
            if (szn >= 0) cpml4(psz + 2 * p.sz + (szn * p.NY + j) * pitch + i, bz, az, dHy_dz);
            const float4 c = ld4(cE + idx);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (vx[e]) at(eo, e) = get(eo, e) + get(c, e) * (get(dHz_dy, e) - get(dHy_dz, e));
        }
        st4(En + idx, eo);
        eo = ld4(Eo + vol + idx);
        if (kin) {                                                // Ey at (i, j+1/2, k)
            float4 dHx_dz = mul(sub(hxc, hxm), ihz), dHz_dx = mul(sub(hzc, hzx), ihx4);
            if (szn >= 0) cpml4(psz + 3 * p.sz + (szn * p.NY + j) * pitch + i, bz, az, dHx_dz);
            if (xslab) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ix = vyz[e] ? slab_node(i + e, nx, npml) : -1;
                    if (ix < 0) continue;
                    float &ps = psx[2 * p.sx + (k * p.NY + j) * np2 + ix];
                    ps = __ldg(p.ax.b_n + i + e) * ps + __ldg(p.ax.a_n + i + e) * get(dHz_dx, e);
                    at(dHz_dx, e) += ps;
                }
            }
            const float4 c = ld4(cE + vol + idx);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (vyz[e]) at(eo, e) = get(eo, e) + get(c, e) * (get(dHx_dz, e) - get(dHz_dx, e));
        }
        st4(En + vol + idx, eo);
        eo = ld4(Eo + 2 * vol + idx);
        if (jin) {                                                // Ez at (i, j, k+1/2)
            float4 dHy_dx = mul(sub(hyc, hyx), ihx4), dHx_dy = mul(sub(hxc, hxj), ihy);
            if (syn >= 0) cpml4(psy + 3 * p.sy + (k * np2 + syn) * pitch + i, by, ay, dHx_dy);
            if (xslab) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ix = vyz[e] ? slab_node(i + e, nx, npml) : -1;
                    if (ix < 0) continue;
                    float &ps = psx[3 * p.sx + (k * p.NY + j) * np2 + ix];
                    ps = __ldg(p.ax.b_n + i + e) * ps + __ldg(p.ax.a_n + i + e) * get(dHy_dx, e);
                    at(dHy_dx, e) += ps;
                }
            }
            const float4 c = ld4(cE + 2 * vol + idx);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (vyz[e]) at(eo, e) = get(eo, e) + get(c, e) * (get(dHy_dx, e) - get(dHx_dy, e));
        }
        st4(En + 2 * vol + idx, eo);
        hxm = hxc;
        hym = hyc;
    }
    // source term E^{n+1} -= dt/eps J'^{n+1/2} for the taps of this thread's four columns
    if (p.colmap) {
        for (int e = 0; e < 4; ++e) {
            if (i + e >= nx) break;
            const int2 cm = p.colmap[s * p.colmap_stride + j * pitch + i + e];
            for (int u = cm.x; u < cm.x + cm.y; ++u) {
                const Tap tp = p.itaps[(long long)s * p.itap_stride + u];
                const int k = (int)(tp.idx / plane);
                if (k < k0 || k >= k1) continue;
                const double *cf = p.coef + ((long long)s * p.n_emit + tp.emit) * p.J;
                const double *T = p.T + (long long)n * p.J;
                double amp = 0.0;
                for (int jj = 0; jj < p.J; ++jj) amp += cf[jj] * T[jj];
                const int o = tp.comp * vol + (int)tp.idx;
                const double add = -(double)p.cE[o] * tp.w * amp;
                if (add != 0.0) En[o] += (float)add;
            }
        }
    }
}

template <int KZ, int MB>
void launch_vec_kz(const StepParams<float> &p, dim3 grid, int jstep, cudaStream_t st, bool h) {
    if (h) k_h4<KZ, MB><<<grid, kBlock, 0, st>>>(p, jstep);
    else k_e4<KZ, MB><<<grid, kBlock, 0, st>>>(p, jstep);
}

cudaError_t launch_field_vec(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int kz, int mb) {
    const long long quads = (long long)p.ny * (p.pitch >> 2);
    dim3 grid((unsigned)((quads + kBlock - 1) / kBlock), (unsigned)((p.nz + kz - 1) / kz), (unsigned)S);
    bool ok = true;
    if (mb == 4) {
        if (kz == 1) launch_vec_kz<1, 4>(p, grid, jstep, st, h);
        else if (kz == 2) launch_vec_kz<2, 4>(p, grid, jstep, st, h);
        else if (kz == 4) launch_vec_kz<4, 4>(p, grid, jstep, st, h);
        else if (kz == 8) launch_vec_kz<8, 4>(p, grid, jstep, st, h);
        else ok = false;
    } else if (mb == 6) {
        if (kz == 1) launch_vec_kz<1, 6>(p, grid, jstep, st, h);
        else if (kz == 2) launch_vec_kz<2, 6>(p, grid, jstep, st, h);
        else if (kz == 4) launch_vec_kz<4, 6>(p, grid, jstep, st, h);
        else if (kz == 8) launch_vec_kz<8, 6>(p, grid, jstep, st, h);
        else ok = false;
    } else {
        ok = false;
    }
    if (!ok) return cudaErrorInvalidValue;
    g_launches++;
    return cudaGetLastError();
}

}  // namespace csem
