// Lean FP32 H and E step kernels (Sec. 2, Eq. 4 with the unsplit CPML): W
// consecutive cells (W = 1 or 2; i a multiple of W) of one (j, k) row per
// thread, the cell range [0,nx) x [0,ny) x [0,nz) (nx a multiple of 4), KZ
// planes along z per thread.  They compute what the scalar kernels compute,
// entry by entry, with every load of a plane independent of the others, so that
// a plane's loads are in flight together:
//  * the CPML memory lives in arrays of its own (12 per source: 0-5 for H, 6-11
//    for E).  The y- and z-slab arrays have the field layout.  The x-slab arrays
//    (3, 4, 9, 10) are compact: row (k, j) holds the 2*nxs cells i < nxs and
//    i >= nx - nxs (nxs = npml rounded up to even), so the slab entries of
//    consecutive rows are contiguous;
//  * the coefficient tables are padded to whole 16-byte groups, and the CPML
//    coefficients are zero off the slabs and on the outer nodes.  A cell in the
//    rounded-out slab but not in the CPML keeps psi = 0;
//  * the x-slab recursion runs on every lane (lanes off the slab read zeros and
//    have zero coefficients) and only slab lanes store, so warps do not diverge
//    on it;
//  * a block whose plane is off the z slabs and whose rows are off the y slabs
//    takes a code path without the y/z recursion, with fewer live values;
//  * E is advanced with dt/eps set to zero on the PEC edges (tangential E on the
//    outer faces), so all three components are written unconditionally, the PEC
//    edges keep their zero, and the curl's lower neighbours are clamped to the
//    cell itself on the outer faces (what they give there is multiplied by 0);
//  * the source taps of the thread's columns are added to the new values in
//    registers before the store; the column map is read only where a per-row,
//    per-32-column flag marks a tap (a byte shared by a warp), inside that rare
//    branch, so it holds no registers elsewhere.
// W stays small so that a plane's loaded values fit the register budget.
// The block is 32 x 4 threads (32 W cells of 4 rows; 128 threads, so 4, 6 or 8
// resident blocks per SM give 128, 85 or 64 registers per thread); blockIdx.z
// runs over (z block, source) with the source fastest.
#include "csem_internal.cuh"

namespace csem {

namespace {

constexpr int kLeanX = 32, kLeanRows = 4;

template <int W> struct Vec { float v[W]; };
template <int W> __device__ __forceinline__ Vec<W> ldc(const float *p) {
    Vec<W> r;
    if constexpr (W == 1) r.v[0] = __ldg(p);
    else { const float2 t = __ldg(reinterpret_cast<const float2 *>(p)); r.v[0] = t.x; r.v[1] = t.y; }
    return r;
}
template <int W> __device__ __forceinline__ Vec<W> ldw(const float *p) {
    Vec<W> r;
    if constexpr (W == 1) r.v[0] = *p;
    else { const float2 t = *reinterpret_cast<const float2 *>(p); r.v[0] = t.x; r.v[1] = t.y; }
    return r;
}
template <int W> __device__ __forceinline__ void stv(float *p, const Vec<W> &a) {
    if constexpr (W == 1) *p = a.v[0];
    else *reinterpret_cast<float2 *>(p) = make_float2(a.v[0], a.v[1]);
}
template <int W> __device__ __forceinline__ Vec<W> zv() {
    Vec<W> r;
#pragma unroll
    for (int e = 0; e < W; ++e) r.v[e] = 0.f;
    return r;
}
// (a - b) * s
template <int W> __device__ __forceinline__ Vec<W> dsc(const Vec<W> &a, const Vec<W> &b, float s) {
    Vec<W> r;
#pragma unroll
    for (int e = 0; e < W; ++e) r.v[e] = (a.v[e] - b.v[e]) * s;
    return r;
}
template <int W> __device__ __forceinline__ Vec<W> dsc(const Vec<W> &a, const Vec<W> &b, const Vec<W> &s) {
    Vec<W> r;
#pragma unroll
    for (int e = 0; e < W; ++e) r.v[e] = (a.v[e] - b.v[e]) * s.v[e];
    return r;
}
// CPML recursion psi <- b psi + a d, then d += psi (shared or per-cell b, a)
template <int W> __device__ __forceinline__ void cpml(Vec<W> &ps, Vec<W> &d, float b, float a) {
#pragma unroll
    for (int e = 0; e < W; ++e) { ps.v[e] = b * ps.v[e] + a * d.v[e]; d.v[e] += ps.v[e]; }
}
template <int W> __device__ __forceinline__ void cpml(Vec<W> &ps, Vec<W> &d, const Vec<W> &b, const Vec<W> &a) {
#pragma unroll
    for (int e = 0; e < W; ++e) { ps.v[e] = b.v[e] * ps.v[e] + a.v[e] * d.v[e]; d.v[e] += ps.v[e]; }
}
// h -= c (u - v)
template <int W> __device__ __forceinline__ void hsub(Vec<W> &h, float c, const Vec<W> &u, const Vec<W> &v) {
#pragma unroll
    for (int e = 0; e < W; ++e) h.v[e] -= c * (u.v[e] - v.v[e]);
}
// eo + c (u - v)
template <int W>
__device__ __forceinline__ Vec<W> eadv(const Vec<W> &eo, const Vec<W> &c, const Vec<W> &u, const Vec<W> &v) {
    Vec<W> r;
#pragma unroll
    for (int e = 0; e < W; ++e) r.v[e] = eo.v[e] + c.v[e] * (u.v[e] - v.v[e]);
    return r;
}
// the W cells shifted by one: (prev, a0, .., a_{W-2}) and (a1, .., a_{W-1}, next)
template <int W> __device__ __forceinline__ Vec<W> down(float prev, const Vec<W> &a) {
    Vec<W> r;
    r.v[0] = prev;
#pragma unroll
    for (int e = 1; e < W; ++e) r.v[e] = a.v[e - 1];
    return r;
}
template <int W> __device__ __forceinline__ Vec<W> up(const Vec<W> &a, float next) {
    Vec<W> r;
#pragma unroll
    for (int e = 0; e + 1 < W; ++e) r.v[e] = a.v[e + 1];
    r.v[W - 1] = next;
    return r;
}

// Per-thread constants shared by the planes of a lean kernel.
template <int W> struct LeanRow {
    int i, j, nxs, ixs;
    bool xs, ys;
    Vec<W> ihx, bx, ax;
    float ihy, by, ay;
};
template <int W>
__device__ __forceinline__ void lean_row(const StepParams<float> &p, const AxisTab<float> &tx, const AxisTab<float> &ty,
                                         bool half, int i, int j, LeanRow<W> &r) {
    const int npml = p.npml;
    r.i = i; r.j = j;
    r.nxs = (npml + 1) & ~1;
    r.xs = (i < r.nxs) || (i + W > p.nx - r.nxs);
    r.ixs = (i < r.nxs) ? i : i - (p.nx - 2 * r.nxs);
    r.ihx = ldc<W>((half ? tx.ih_h : tx.ih_n) + i);
    r.bx = ldc<W>((half ? tx.b_h : tx.b_n) + i);
    r.ax = ldc<W>((half ? tx.a_h : tx.a_n) + i);
    r.ihy = __ldg((half ? ty.ih_h : ty.ih_n) + j);
    r.ys = half ? ((j < npml) || (j >= p.ny - npml)) : ((j < npml) || (j > p.ny - npml));
    r.by = r.ys ? __ldg((half ? ty.b_h : ty.b_n) + j) : 0.f;
    r.ay = r.ys ? __ldg((half ? ty.a_h : ty.a_n) + j) : 0.f;
}

// Source term E^{n+1} -= dt/eps J'^{n+1/2} for the taps in plane k of one
// column (first tap, count in cm): the increments were computed for the chunk's
// steps by k_tap_inc, so each tap costs two independent loads.
__device__ __forceinline__ float3 lean_taps(const int *__restrict__ tk, const float *__restrict__ inc, int k, int2 cm) {
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

}  // namespace

// One plane k of the H update for the thread's W cells; YZ: the y/z recursion
// may apply (a block on a y or z slab).  exc, eyc: Ex, Ey of plane k (in), of
// plane k+1 (out).
template <int W, bool YZ>
__device__ __forceinline__ void h_plane(const StepParams<float> &p, const float *__restrict__ E, float *__restrict__ H,
                                        float *__restrict__ ps, const LeanRow<W> &r, int k, int idx, Vec<W> &exc,
                                        Vec<W> &eyc) {
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch, npml = p.npml;
    const Vec<W> ezc = ldc<W>(E + 2 * vol + idx);
    const Vec<W> exk = ldc<W>(E + idx + plane), eyk = ldc<W>(E + vol + idx + plane);
    const Vec<W> exj = ldc<W>(E + idx + pitch), ezj = ldc<W>(E + 2 * vol + idx + pitch);
    const float eyn = __ldg(E + vol + idx + W), ezn = __ldg(E + 2 * vol + idx + W);
    const float ihz = __ldg(p.lz.ih_h + k);
    Vec<W> hx = ldw<W>(H + idx), hy = ldw<W>(H + vol + idx), hz = ldw<W>(H + 2 * vol + idx);
    const int xo = (k * p.ny + r.j) * (2 * r.nxs) + r.ixs;
    float *px3 = ps + 3 * vol + xo, *px4 = ps + 4 * vol + xo;
    Vec<W> q3 = ldw<W>(r.xs ? px3 : p.lzero), q4 = ldw<W>(r.xs ? px4 : p.lzero);
    bool zs = false, ys = false;
    float bz = 0.f, az = 0.f;
    Vec<W> q0 = zv<W>(), q1 = zv<W>(), q2 = zv<W>(), q5 = zv<W>();
    if constexpr (YZ) {
        zs = (k < npml) || (k >= p.nz - npml);
        ys = r.ys;
        if (zs) { bz = __ldg(p.lz.b_h + k); az = __ldg(p.lz.a_h + k); }
        if (ys) { q0 = ldw<W>(ps + idx); q5 = ldw<W>(ps + 5 * vol + idx); }
        if (zs) { q1 = ldw<W>(ps + vol + idx); q2 = ldw<W>(ps + 2 * vol + idx); }
    }
    const Vec<W> ezx = up<W>(ezc, ezn), eyx = up<W>(eyc, eyn);   // Ez, Ey at i+1 .. i+W

    // Hx at (i, j+1/2, k+1/2)
    Vec<W> dEz_dy = dsc<W>(ezj, ezc, r.ihy), dEy_dz = dsc<W>(eyk, eyc, ihz);
    if (YZ && ys) { cpml<W>(q0, dEz_dy, r.by, r.ay); stv<W>(ps + idx, q0); }
    if (YZ && zs) { cpml<W>(q1, dEy_dz, bz, az); stv<W>(ps + vol + idx, q1); }
    hsub<W>(hx, p.cH, dEz_dy, dEy_dz);
    // Hy at (i+1/2, j, k+1/2)
    Vec<W> dEx_dz = dsc<W>(exk, exc, ihz), dEz_dx = dsc<W>(ezx, ezc, r.ihx);
    if (YZ && zs) { cpml<W>(q2, dEx_dz, bz, az); stv<W>(ps + 2 * vol + idx, q2); }
    cpml<W>(q3, dEz_dx, r.bx, r.ax);
    if (r.xs) stv<W>(px3, q3);
    hsub<W>(hy, p.cH, dEx_dz, dEz_dx);
    // Hz at (i+1/2, j+1/2, k)
    Vec<W> dEy_dx = dsc<W>(eyx, eyc, r.ihx), dEx_dy = dsc<W>(exj, exc, r.ihy);
    cpml<W>(q4, dEy_dx, r.bx, r.ax);
    if (r.xs) stv<W>(px4, q4);
    if (YZ && ys) { cpml<W>(q5, dEx_dy, r.by, r.ay); stv<W>(ps + 5 * vol + idx, q5); }
    hsub<W>(hz, p.cH, dEy_dx, dEx_dy);

    stv<W>(H + idx, hx);
    stv<W>(H + vol + idx, hy);
    stv<W>(H + 2 * vol + idx, hz);
    exc = exk;
    eyc = eyk;
}

// H over the KZ planes from z block kb of the tile (xb, yb) of source s (the tile: 32 W
// cells of 4 rows, one W-cell column per thread): k_h_lean's block with its coordinates
// as arguments, for the wave-ordered step (k_h_lean keeps its own copy, compiled as tuned).
template <int W, int KZ>
__device__ __forceinline__ void h_tile(const StepParams<float> &p, const int jstep, int xb, int yb, int kb, int s) {
    const int i = (xb * kLeanX + (int)threadIdx.x) * W;
    const int j = yb * kLeanRows + (int)threadIdx.y;
    const int k0 = kb * KZ;
    if (i >= p.nx || j >= p.ny) return;
    const int k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int vol = (int)p.vol, plane = (int)p.plane, npml = p.npml;
    const float *__restrict__ E = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    float *__restrict__ H = p.H + (long long)s * 3 * vol;
    float *__restrict__ ps = p.psiL + (long long)s * 12 * vol;
    LeanRow<W> r;
    lean_row<W>(p, p.lx, p.ly, true, i, j, r);
    const int j0 = yb * kLeanRows;
    const bool yblk = (j0 < npml) || (j0 + kLeanRows > p.ny - npml);

    int idx = k0 * plane + j * p.pitch + i;
    Vec<W> exc = ldc<W>(E + idx), eyc = ldc<W>(E + vol + idx);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= k1) break;
        if (yblk || k < npml || k >= p.nz - npml) h_plane<W, true>(p, E, H, ps, r, k, idx, exc, eyc);
        else h_plane<W, false>(p, E, H, ps, r, k, idx, exc, eyc);
    }
}

template <int W, int KZ, int MINB>
__global__ void __launch_bounds__(kLeanX *kLeanRows, MINB) k_h_lean(const StepParams<float> p, const int jstep) {
    const int i = (blockIdx.x * kLeanX + threadIdx.x) * W;
    const int j = blockIdx.y * kLeanRows + threadIdx.y;
    const int nkb = (p.nz + KZ - 1) / KZ;
    const int S = gridDim.z / nkb;
    const int s = blockIdx.z % S;                 // the source runs fastest: the sources of one
    const int k0 = (blockIdx.z / S) * KZ;         // z block follow one another
    if (i >= p.nx || j >= p.ny) return;
    const int k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int vol = (int)p.vol, plane = (int)p.plane, npml = p.npml;
    const float *__restrict__ E = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    float *__restrict__ H = p.H + (long long)s * 3 * vol;
    float *__restrict__ ps = p.psiL + (long long)s * 12 * vol;
    LeanRow<W> r;
    lean_row<W>(p, p.lx, p.ly, true, i, j, r);
    const int j0 = blockIdx.y * kLeanRows;
    const bool yblk = (j0 < npml) || (j0 + kLeanRows > p.ny - npml);

    int idx = k0 * plane + j * p.pitch + i;
    Vec<W> exc = ldc<W>(E + idx), eyc = ldc<W>(E + vol + idx);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= k1) break;
        if (yblk || k < npml || k >= p.nz - npml) h_plane<W, true>(p, E, H, ps, r, k, idx, exc, eyc);
        else h_plane<W, false>(p, E, H, ps, r, k, idx, exc, eyc);
    }
}

// H loads of the E update: through the read-only path, or (CG) from L2 only, for H that
// other blocks of the same launch wrote (the read-only path and L1 are not coherent with them).
template <int W, bool CG> __device__ __forceinline__ Vec<W> ldh(const float *p) {
    if constexpr (!CG) return ldc<W>(p);
    Vec<W> r;
    if constexpr (W == 1) r.v[0] = __ldcg(p);
    else { const float2 t = __ldcg(reinterpret_cast<const float2 *>(p)); r.v[0] = t.x; r.v[1] = t.y; }
    return r;
}
template <bool CG> __device__ __forceinline__ float ldh1(const float *p) { return CG ? __ldcg(p) : __ldg(p); }

// One plane k of the E update; hxm, hym: Hx, Hy of plane k-1 (in), of plane k (out).
template <int W, bool YZ, bool CG>
__device__ __forceinline__ void e_plane(const StepParams<float> &p, const float *__restrict__ Eo, float *__restrict__ En,
                                        const float *__restrict__ H, float *__restrict__ ps, const LeanRow<W> &r, int s,
                                        int S, int jstep, int k, int idx, bool taps, Vec<W> &hxm, Vec<W> &hym) {
    const int vol = (int)p.vol, pitch = p.pitch, npml = p.npml;
    const float *__restrict__ cE = p.cEm;
    const int ij = (r.j > 0) ? idx - pitch : idx;    // lower neighbours, clamped on the outer faces
    const int ii = (r.i > 0) ? idx - 1 : idx;
    const Vec<W> hxc = ldh<W, CG>(H + idx), hyc = ldh<W, CG>(H + vol + idx), hzc = ldh<W, CG>(H + 2 * vol + idx);
    const Vec<W> hxj = ldh<W, CG>(H + ij), hzj = ldh<W, CG>(H + 2 * vol + ij);
    const float hyp = ldh1<CG>(H + vol + ii), hzp = ldh1<CG>(H + 2 * vol + ii);
    const Vec<W> eo0 = ldc<W>(Eo + idx), eo1 = ldc<W>(Eo + vol + idx), eo2 = ldc<W>(Eo + 2 * vol + idx);
    const Vec<W> c0 = ldc<W>(cE + idx), c1 = ldc<W>(cE + vol + idx), c2 = ldc<W>(cE + 2 * vol + idx);
    const float ihz = __ldg(p.lz.ih_n + k);
    const int xo = (k * p.ny + r.j) * (2 * r.nxs) + r.ixs;
    float *px3 = ps + 3 * vol + xo, *px4 = ps + 4 * vol + xo;
    Vec<W> q3 = ldw<W>(r.xs ? px3 : p.lzero), q4 = ldw<W>(r.xs ? px4 : p.lzero);
    bool zs = false, ys = false;
    float bz = 0.f, az = 0.f;
    Vec<W> q0 = zv<W>(), q1 = zv<W>(), q2 = zv<W>(), q5 = zv<W>();
    if constexpr (YZ) {
        zs = (k < npml) || (k > p.nz - npml);
        ys = r.ys;
        if (zs) { bz = __ldg(p.lz.b_n + k); az = __ldg(p.lz.a_n + k); }
        if (ys) { q0 = ldw<W>(ps + idx); q5 = ldw<W>(ps + 5 * vol + idx); }
        if (zs) { q1 = ldw<W>(ps + vol + idx); q2 = ldw<W>(ps + 2 * vol + idx); }
    }
    const Vec<W> hzx = down<W>(hzp, hzc), hyx = down<W>(hyp, hyc);   // Hz, Hy at i-1 .. i+W-2

    // Ex at (i+1/2, j, k)
    Vec<W> dHz_dy = dsc<W>(hzc, hzj, r.ihy), dHy_dz = dsc<W>(hyc, hym, ihz);
    if (YZ && ys) { cpml<W>(q0, dHz_dy, r.by, r.ay); stv<W>(ps + idx, q0); }
    if (YZ && zs) { cpml<W>(q1, dHy_dz, bz, az); stv<W>(ps + vol + idx, q1); }
    Vec<W> e0 = eadv<W>(eo0, c0, dHz_dy, dHy_dz);
    // Ey at (i, j+1/2, k)
    Vec<W> dHx_dz = dsc<W>(hxc, hxm, ihz), dHz_dx = dsc<W>(hzc, hzx, r.ihx);
    if (YZ && zs) { cpml<W>(q2, dHx_dz, bz, az); stv<W>(ps + 2 * vol + idx, q2); }
    cpml<W>(q3, dHz_dx, r.bx, r.ax);
    if (r.xs) stv<W>(px3, q3);
    Vec<W> e1 = eadv<W>(eo1, c1, dHx_dz, dHz_dx);
    // Ez at (i, j, k+1/2)
    Vec<W> dHy_dx = dsc<W>(hyc, hyx, r.ihx), dHx_dy = dsc<W>(hxc, hxj, r.ihy);
    cpml<W>(q4, dHy_dx, r.bx, r.ax);
    if (r.xs) stv<W>(px4, q4);
    if (YZ && ys) { cpml<W>(q5, dHx_dy, r.by, r.ay); stv<W>(ps + 5 * vol + idx, q5); }
    Vec<W> e2 = eadv<W>(eo2, c2, dHy_dx, dHx_dy);

    if (taps) {
        const int2 *cm = p.colmap + (long long)s * p.colmap_stride + r.j * pitch + r.i;
        const int *tk = p.tapk + (long long)s * p.itap_stride;
        const float *inc = p.inc + ((long long)jstep * S + s) * p.inc_ntl;
        for (int e = 0; e < W; ++e) {
            const int2 c = __ldg(cm + e);
            if (c.y == 0) continue;
            const float3 a = lean_taps(tk, inc, k, c);
            e0.v[e] += a.x; e1.v[e] += a.y; e2.v[e] += a.z;
        }
    }
    stv<W>(En + idx, e0);
    stv<W>(En + vol + idx, e1);
    stv<W>(En + 2 * vol + idx, e2);
    hxm = hxc;
    hym = hyc;
}

// E over the KZ planes from z block kb of the tile (xb, yb) of source s (S sources per
// launch): k_e_lean's block with its coordinates as arguments, H read through ldh<CG>.
template <int W, int KZ, bool CG>
__device__ __forceinline__ void e_tile(const StepParams<float> &p, const int jstep, int xb, int yb, int kb, int s,
                                       int S) {
    const int i = (xb * kLeanX + (int)threadIdx.x) * W;
    const int j = yb * kLeanRows + (int)threadIdx.y;
    const int k0 = kb * KZ;
    if (i >= p.nx || j >= p.ny) return;
    const int k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch, npml = p.npml;
    const float *__restrict__ ring = p.ering + (long long)s * p.ering_stride;
    const float *__restrict__ Eo = ring + (long long)(n % p.nslot) * 3 * p.vol;
    float *__restrict__ En = const_cast<float *>(ring) + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    const float *__restrict__ H = p.H + (long long)s * 3 * vol;
    float *__restrict__ ps = p.psiL + (long long)s * 12 * vol + 6LL * vol;
    LeanRow<W> r;
    lean_row<W>(p, p.lx, p.ly, false, i, j, r);
    const int j0 = yb * kLeanRows;
    const bool yblk = (j0 < npml) || (j0 + kLeanRows - 1 > p.ny - npml);
    const bool taps = p.colmap && p.inc && p.tflag[s * p.tflag_stride + j * p.nseg + (i >> 5)];

    int idx = k0 * plane + j * pitch + i;
    const int im = (k0 > 0) ? idx - plane : idx;      // clamped on the bottom face
    Vec<W> hxm = ldh<W, CG>(H + im), hym = ldh<W, CG>(H + vol + im);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= k1) break;
        if (yblk || k < npml || k > p.nz - npml)
            e_plane<W, true, CG>(p, Eo, En, H, ps, r, s, S, jstep, k, idx, taps, hxm, hym);
        else e_plane<W, false, CG>(p, Eo, En, H, ps, r, s, S, jstep, k, idx, taps, hxm, hym);
    }
}

template <int W, int KZ, int MINB>
__global__ void __launch_bounds__(kLeanX *kLeanRows, MINB) k_e_lean(const StepParams<float> p, const int jstep) {
    const int i = (blockIdx.x * kLeanX + threadIdx.x) * W;
    const int j = blockIdx.y * kLeanRows + threadIdx.y;
    const int nkb = (p.nz + KZ - 1) / KZ;
    const int S = gridDim.z / nkb;
    const int s = blockIdx.z % S;                 // the source runs fastest: the sources of one z
    const int k0 = (blockIdx.z / S) * KZ;         // block share the dt/eps reads in L2
    if (i >= p.nx || j >= p.ny) return;
    const int k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch, npml = p.npml;
    const float *__restrict__ ring = p.ering + (long long)s * p.ering_stride;
    const float *__restrict__ Eo = ring + (long long)(n % p.nslot) * 3 * p.vol;
    float *__restrict__ En = const_cast<float *>(ring) + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    const float *__restrict__ H = p.H + (long long)s * 3 * vol;
    float *__restrict__ ps = p.psiL + (long long)s * 12 * vol + 6LL * vol;
    LeanRow<W> r;
    lean_row<W>(p, p.lx, p.ly, false, i, j, r);
    const int j0 = blockIdx.y * kLeanRows;
    const bool yblk = (j0 < npml) || (j0 + kLeanRows - 1 > p.ny - npml);
    const bool taps = p.colmap && p.inc && p.tflag[s * p.tflag_stride + j * p.nseg + (i >> 5)];

    int idx = k0 * plane + j * pitch + i;
    const int im = (k0 > 0) ? idx - plane : idx;      // clamped on the bottom face
    Vec<W> hxm = ldc<W>(H + im), hym = ldc<W>(H + vol + im);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= k1) break;
        if (yblk || k < npml || k > p.nz - npml) e_plane<W, true, false>(p, Eo, En, H, ps, r, s, S, jstep, k, idx, taps, hxm, hym);
        else e_plane<W, false, false>(p, Eo, En, H, ps, r, s, S, jstep, k, idx, taps, hxm, hym);
    }
}

// One whole step (H then E) in one launch, ordered by tickets: every block takes the next
// ticket from a counter, and the tickets run through the z blocks ("chunks") as
//   H(0) .. H(lag-1), then H(c + lag), E(c) for c = 0, 1, .., then the remaining E(c),
// each chunk being all tiles of its z block (the sources of a tile next to one another).
// The E tiles of chunk c read H of chunks c and c-1, which the H tiles of those chunks
// write in the same launch: the H tiles count themselves done per chunk (after a fence),
// and an E tile's thread 0 waits (bounded, about a second) until both chunks are complete.
// No H tile waits, and an E tile waits only for tiles that took earlier tickets, so every
// wait ends.  The lag keeps the E tiles far enough behind that the H tiles they need have
// usually finished, and near enough that the E^n and H^{n+1/2} they read were touched a few
// chunks before and are still in L2: that is the point of the ordering -- E reads them
// from L2 instead of DRAM.  H is read from L2 only (__ldcg) by the E tiles.  The last
// block to finish resets the counters, so the next launch starts from zero.
// wave[0]: ticket counter, wave[1]: finished blocks, wave[2 + c]: H tiles done in chunk c.
// Chunks of the wave-ordered step: z blocks, and tiles per z block (every source).
template <int W, int KZ> __device__ __forceinline__ unsigned wave_nkb(const StepParams<float> &p) {
    return (unsigned)((p.nz + KZ - 1) / KZ);
}
template <int W, int KZ> __device__ __forceinline__ unsigned wave_tc(const StepParams<float> &p, int S) {
    return (unsigned)((p.nx / W + kLeanX - 1) / kLeanX) * (unsigned)((p.ny + kLeanRows - 1) / kLeanRows) * (unsigned)S;
}

template <int W, int KZ, int MINB>
__global__ void __launch_bounds__(kLeanX *kLeanRows, MINB) k_step_wave(const StepParams<float> p, const int jstep,
                                                                     const int S, const int lag) {
    __shared__ int tile[5];                        // H (1) or E (0), z block, source, x tile, y tile
    const int tid = threadIdx.y * kLeanX + threadIdx.x;
    if (tid == 0) {                                // thread 0 takes the ticket and decodes it
        const unsigned t = atomicAdd(p.wave, 1u);
        const unsigned nkb = wave_nkb<W, KZ>(p), tc = wave_tc<W, KZ>(p, S);
        const unsigned nxb = (unsigned)((p.nx / W + kLeanX - 1) / kLeanX);
        const unsigned L = (unsigned)min(max(lag, 1), (int)nkb);
        bool h;
        unsigned kb, r;
        if (t < L * tc) {
            h = true; kb = t / tc; r = t % tc;
        } else {
            const unsigned u = t - L * tc, mid = (nkb - L) * 2u * tc;
            if (u < mid) {
                const unsigned ph = u / (2u * tc), q = u % (2u * tc);
                h = q < tc;
                kb = h ? L + ph : ph;
                r = h ? q : q - tc;
            } else {
                h = false; kb = (nkb - L) + (u - mid) / tc; r = (u - mid) % tc;
            }
        }
        tile[0] = h ? 1 : 0;
        tile[1] = (int)kb;
        tile[2] = (int)(r % (unsigned)S);
        tile[3] = (int)((r / (unsigned)S) % nxb);
        tile[4] = (int)(r / ((unsigned)S * nxb));
        if (!h) {                                  // E: wait until H of z blocks kb and kb - 1 is complete
            // the test hook makes the wait unsatisfiable; once one wait gave up, the others skip it
            const unsigned need = tc + (p.fault_tx ? 1u : 0u);
            const unsigned *done = p.wave + 2;
            const unsigned long long t0 = gtimer_ns();
            for (unsigned it = 0;; ++it) {
                const unsigned a = *(volatile const unsigned *)&done[kb];
                const unsigned b = kb ? *(volatile const unsigned *)&done[kb - 1] : need;
                if (a >= need && b >= need) break;
                if ((*(volatile int *)p.err) & kErrWaveWait) break;
                if (it >= (1u << 24) || ((it & 63) == 63 && gtimer_ns() - t0 > kWaitNs)) {
                    atomicOr(p.err, kErrWaveWait);
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
    }
    __syncthreads();
    if (tile[0]) {
        h_tile<W, KZ>(p, jstep, tile[3], tile[4], tile[1], tile[2]);
        __syncthreads();
        if (tid == 0) {
            __threadfence();                       // the block's H stores before the count
            atomicAdd(p.wave + 2 + tile[1], 1u);
        }
    } else {
        e_tile<W, KZ, true>(p, jstep, tile[3], tile[4], tile[1], tile[2], S);
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned nkb = wave_nkb<W, KZ>(p);
        if (atomicAdd(p.wave + 1, 1u) == 2u * nkb * wave_tc<W, KZ>(p, S) - 1u) {   // all others finished
            p.wave[0] = 0u;
            p.wave[1] = 0u;
            for (unsigned c = 0; c < nkb; ++c) p.wave[2 + c] = 0u;
            __threadfence();
        }
    }
}

// Increment -dt/eps J'^{n+1/2} of every injection tap (Sec. 2, Eq. 4 source
// term; the amplitude sum_j coef_j T_j(n) in FP64, one rounding to FP32, the same
// value the other step kernels add) for the steps jstep in [0, nsteps) after the
// device step counter: inc[(jstep*S + s)*inc_ntl + u].
__global__ void k_tap_inc(const StepParams<float> p, const int S, const int nsteps, const int nt) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ntl = p.inc_ntl;
    if (t >= (long long)nsteps * S * ntl) return;
    const int u = (int)(t % ntl);
    const int s = (int)((t / ntl) % S);
    const int jstep = (int)(t / ((long long)ntl * S));
    const int n = *p.step + jstep;
    float v = 0.f;
    if (n < nt) {
        const Tap tp = p.itaps[(long long)s * p.itap_stride + u];
        const double *cf = p.coef + ((long long)s * p.n_emit + tp.emit) * p.J;
        const double *T = p.T + (long long)n * p.J;
        double amp = 0.0;
        for (int jj = 0; jj < p.J; ++jj) amp += cf[jj] * T[jj];
        const int o = tp.comp * (int)p.vol + (int)tp.idx;
        v = (float)(-(double)p.cE[o] * tp.w * amp);
    }
    p.inc[t] = v;
}

// dt/eps with the PEC edges zeroed: Ex needs 1 <= j < ny, 1 <= k < nz, i < nx;
// Ey 1 <= i < nx, 1 <= k < nz, j < ny; Ez 1 <= i < nx, 1 <= j < ny, k < nz.
__global__ void k_mask_coef(const StepParams<float> p, const float *__restrict__ cE, float *__restrict__ cEm) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * p.vol) return;
    const int c = (int)(t / p.vol);
    const int idx = (int)(t - (long long)c * p.vol);
    const int k = idx / (int)p.plane;
    const int r = idx - k * (int)p.plane;
    const int j = r / p.pitch;
    const int i = r - j * p.pitch;
    const bool xi = (i >= 1 && i < p.nx), yi = (j >= 1 && j < p.ny), zi = (k >= 1 && k < p.nz);
    bool ok;
    if (c == 0) ok = (i < p.nx) && yi && zi;
    else if (c == 1) ok = xi && (j < p.ny) && zi;
    else ok = xi && yi && (k < p.nz);
    cEm[t] = ok ? cE[t] : 0.f;
}

namespace {
template <int W, int KZ, int MB>
void lean_go(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h) {
    const dim3 block(kLeanX, kLeanRows);
    const int nv = p.nx / W;
    const dim3 grid((nv + kLeanX - 1) / kLeanX, (p.ny + kLeanRows - 1) / kLeanRows, ((p.nz + KZ - 1) / KZ) * S);
    if (h) k_h_lean<W, KZ, MB><<<grid, block, 0, st>>>(p, jstep);
    else k_e_lean<W, KZ, MB><<<grid, block, 0, st>>>(p, jstep);
}
template <int W, int MB>
bool lean_kz(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int kz) {
    switch (kz) {
        case 1: lean_go<W, 1, MB>(p, S, jstep, st, h); return true;
        case 2: lean_go<W, 2, MB>(p, S, jstep, st, h); return true;
        case 4: lean_go<W, 4, MB>(p, S, jstep, st, h); return true;
        default: return false;
    }
}
}  // namespace

cudaError_t launch_field_lean(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int w, int kz,
                              int mb) {
    if (p.nx % 4 != 0 || !p.psiL || !p.cEm || !p.lx.ih_n || !p.lzero) return cudaErrorInvalidValue;
    bool ok = false;
    if (w == 1 && mb == 6) ok = lean_kz<1, 6>(p, S, jstep, st, h, kz);
    else if (w == 1 && mb == 8) ok = lean_kz<1, 8>(p, S, jstep, st, h, kz);
    else if (w == 2 && mb == 4) ok = lean_kz<2, 4>(p, S, jstep, st, h, kz);
    else if (w == 2 && mb == 6) ok = lean_kz<2, 6>(p, S, jstep, st, h, kz);
    else if (w == 2 && mb == 8) ok = lean_kz<2, 8>(p, S, jstep, st, h, kz);
    if (!ok) return cudaErrorInvalidValue;
    g_launches++;
    return cudaGetLastError();
}

bool wave_supported(const StepParams<float> &p, int kz, int mb) {
    return p.wave && p.nx % 4 == 0 && p.psiL && p.cEm && p.lx.ih_n && p.lzero && (kz == 2 || kz == 4) &&
           (mb == 6 || mb == 8) && p.nz <= kMaxWaveChunks * kz;
}

cudaError_t launch_step_wave(const StepParams<float> &p, int S, int jstep, cudaStream_t st) {
    const int kz = p.WAVE_kz, mb = p.WAVE_mb, lag = p.WAVE_lag;
    if (!wave_supported(p, kz, mb) || lag < 1) return cudaErrorInvalidValue;
    const long long nxb = (p.nx / 2 + kLeanX - 1) / kLeanX, nyb = (p.ny + kLeanRows - 1) / kLeanRows;
    const long long nblk = 2LL * ((p.nz + kz - 1) / kz) * nxb * nyb * S;
    const dim3 block(kLeanX, kLeanRows);
    if (kz == 2 && mb == 6) k_step_wave<2, 2, 6><<<(unsigned)nblk, block, 0, st>>>(p, jstep, S, lag);
    else if (kz == 2) k_step_wave<2, 2, 8><<<(unsigned)nblk, block, 0, st>>>(p, jstep, S, lag);
    else if (mb == 6) k_step_wave<2, 4, 6><<<(unsigned)nblk, block, 0, st>>>(p, jstep, S, lag);
    else k_step_wave<2, 4, 8><<<(unsigned)nblk, block, 0, st>>>(p, jstep, S, lag);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_tap_inc(const StepParams<float> &p, int S, int nsteps, int nt, cudaStream_t st) {
    const long long n = (long long)nsteps * S * p.inc_ntl;
    if (n <= 0 || !p.inc || !p.itaps) return cudaSuccess;
    k_tap_inc<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, S, nsteps, nt);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_mask_coef(const StepParams<float> &p, const float *cE, float *cEm, cudaStream_t st) {
    const long long n = 3 * p.vol;
    k_mask_coef<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, cE, cEm);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace csem
