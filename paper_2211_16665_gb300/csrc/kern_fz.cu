// Fused FP32 leap-frog step that reads every field once per step (Sec. 2,
// Eq. 4, with the unsplit CPML): H^{n-1/2} -> H^{n+1/2} and E^n -> E^{n+1} in
// one kernel, source injection included.
//
// A block of 32 x (BY + 1) threads owns a tile of 64 cells (x) by BY rows (y)
// and marches KZ planes along z; each of the first BY warps owns one row, each
// thread two consecutive cells (i, i+1) of it; the last warp is the halo warp.  The planes are staged into shared memory by the tensor memory
// accelerator: one thread issues, per plane m, three 4-D tile copies -- E^n
// (Ex, Ey, Ez), H^{n-1/2} (Hx, Hy, Hz) and the per-cell material -- each 72
// columns (x from i0-4, so the copy starts on a 16-byte boundary) by BY+2 rows
// (y from j0-1) of plane m, into a ring of NST stages with one mbarrier each.
// Coordinates outside the lattice (the faces of the grid, ragged tiles) are
// filled with zeros by the copy engine.  Planes m+1 .. m+NST-2 are in flight
// while plane m is computed, so the DRAM latency is hidden by the ring rather
// than by resident warps.  Per plane k, from shared memory:
//  * phase 1: H^{n+1/2} of every thread's two cells into a shared plane (and to
//    the second H buffer in global memory); the halo warp computes H^{n+1/2} of
//    row j0-1 and, lane by lane, Hy and Hz of column i0-1 -- values the
//    neighbouring blocks own, recomputed from the staged E^n and H^{n-1/2}
//    rather than exchanged, so no block waits on another or reads a value
//    another block has advanced.  H and the CPML memory of the H update are
//    double buffered (step n reads the buffer of parity n and writes the
//    other), E^n and E^{n+1} are different ring slots, and the CPML memory of
//    the E update is touched only by the cell's owner;
//  * phase 2, after a block barrier: E^{n+1} of the thread's cells with the
//    neighbouring H values (i-1, j-1) from the shared plane and those of
//    plane k-1 kept in registers;
//  * dt/eps on the three edges of the node comes from one value per cell,
//    q = V sigma (cell volume times conductivity): the edge conductivity is the
//    volume-weighted mean of the four cells around the edge, so dt/eps = 2 w0 dt
//    (sum of the four volumes) / (sum of the four q), the volume sum a product
//    of one width per axis (a VTI medium stages sigma_v as a second value for
//    its z edges);
//  * the PEC edges (tangential E on the outer faces) get a zero coefficient,
//    so all three components are stored unconditionally;
//  * the CPML memory (inside the slabs only) is read and written directly;
//  * the source taps of the thread's columns are added from the per-chunk tap
//    increments, read only where the per-row, per-32-column flag marks a tap.
// A z block that starts at k0 > 0 first recomputes Hx, Hy of plane k0-1 (the
// block below owns and writes them).  blockIdx.x runs over (x tile, source)
// with the source fastest, so the blocks of all sources of one tile run close
// together and share the material reads in L2.
//
// Every wait on a stage barrier is bounded (about a second): a block that gives
// up leaves the plane loop with all its threads together, raises the one-pass
// bit of *err, waits (again bounded) for the copies it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "csem_internal.cuh"

namespace csem {

namespace {

constexpr int kXW = 72;            // staged columns: x from i0 - 4 to i0 + 67

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void fz_bar_init(uint64_t *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(b)) : "memory");
}
__device__ __forceinline__ void fz_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void fz_tile4(void *dst, const CUtensorMap *m, int x, int y, int z, int w, uint64_t *b) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(s_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(m)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(s_u32(b))
        : "memory");
}
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 dsc(float2 a, float2 b, float s) { return f2((a.x - b.x) * s, (a.y - b.y) * s); }
__device__ __forceinline__ float2 dsc(float2 a, float2 b, float2 s) { return f2((a.x - b.x) * s.x, (a.y - b.y) * s.y); }
// psi <- b psi + a d; d += psi
__device__ __forceinline__ void rec2(float2 &ps, float2 &d, float b, float a) {
    ps.x = b * ps.x + a * d.x; ps.y = b * ps.y + a * d.y;
    d.x += ps.x; d.y += ps.y;
}
__device__ __forceinline__ void rec1(float &ps, float &d, float b, float a) {
    ps = b * ps + a * d;
    d += ps;
}
// h - c (u - v)
__device__ __forceinline__ float2 hupd(float2 h, float c, float2 u, float2 v) {
    return f2(h.x - c * (u.x - v.x), h.y - c * (u.y - v.y));
}

// Source term of one column: the increments -dt/eps J'^{n+1/2} of its taps in plane k.
__device__ __forceinline__ float3 taps_at(const int *__restrict__ tk, const float *__restrict__ inc, int k, int2 cm) {
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

// A stage holds plane m as three blocks, each starting on a 128-byte boundary: E (Ex, Ey, Ez),
// H (Hx, Hy, Hz) and nq material values, every component (by+2) rows of kXW floats, dense
// within its block (one tile copy writes a block).
__host__ __device__ inline int fz_r32(int f) { return (f + 31) / 32 * 32; }
__host__ __device__ inline int fz_block3(int by) { return fz_r32(3 * (by + 2) * kXW); }
__host__ __device__ inline int fz_stage_floats(int by, int nq) { return 2 * fz_block3(by) + fz_r32(nq * (by + 2) * kXW); }

// per-plane z tables staged in shared memory at block start
struct ZT {
    float ihzh, ihzn, bzh, azh, bzn, azn, gzh, gzs;
    int szh, szn, pad0, pad1;      // slab indices of the half node and the node k (-1 off the slabs)
};
// stages of the plane ring per launch shape (shared memory allows 3 for the denser shapes)
__host__ __device__ constexpr int fz_nst(int by, int mb) { return (by == 4 && mb == 6) || (by == 8 && mb == 3) ? 3 : 4; }

// x-axis constants of a cell pair (i, i+1) for the H update (half nodes)
struct XH {
    float2 ih;
    float b0, a0, b1, a1;
    int s0, s1;
};
// y-axis constants of a row j for the H update
struct YH {
    float ih, b, a;
    int s;
};
__device__ __forceinline__ XH xh_of(const StepParams<float> &p, int i) {
    XH x;
    x.ih = *reinterpret_cast<const float2 *>(p.lx.ih_h + i);
    x.b0 = __ldg(p.lx.b_h + i); x.a0 = __ldg(p.lx.a_h + i);
    x.b1 = __ldg(p.lx.b_h + i + 1); x.a1 = __ldg(p.lx.a_h + i + 1);
    x.s0 = slab_half(i, p.nx, p.npml); x.s1 = slab_half(i + 1, p.nx, p.npml);
    return x;
}
__device__ __forceinline__ YH yh_of(const StepParams<float> &p, int j) {
    YH y;
    y.ih = __ldg(p.ly.ih_h + j); y.b = __ldg(p.ly.b_h + j); y.a = __ldg(p.ly.a_h + j);
    y.s = slab_half(j, p.ny, p.npml);
    return y;
}

// H^{n+1/2} of the cell pair (i, i+1) of row j, plane k, from the staged planes S0 (k) and
// S1 (k+1) at offset o of the pair's first cell; the CPML memory of the H update is read from
// buffer hin and, when wr, written to buffer hout.
__device__ __forceinline__ void h_pair(const StepParams<float> &p, const float *S0, const float *S1, int B3, int PL,
                                       int o, int i, int j, int k, int szh, const ZT &z, const XH &xh, const YH &yh,
                                       bool wr, float *P, int hin, int hout, float2 &hx, float2 &hy, float2 &hz) {
    const float *Ex0 = S0, *Ey0 = S0 + PL, *Ez0 = S0 + 2 * PL;
    const float2 ex = ld2(Ex0 + o), ey = ld2(Ey0 + o), ez = ld2(Ez0 + o);
    float2 dEz_dy = dsc(ld2(Ez0 + o + kXW), ez, yh.ih), dEy_dz = dsc(ld2(S1 + PL + o), ey, z.ihzh);
    float2 dEx_dz = dsc(ld2(S1 + o), ex, z.ihzh), dEz_dx = dsc(f2(ez.y, Ez0[o + 2]), ez, xh.ih);
    float2 dEy_dx = dsc(f2(ey.y, Ey0[o + 2]), ey, xh.ih), dEx_dy = dsc(ld2(Ex0 + o + kXW), ex, yh.ih);
    const int pitch = p.pitch, NY = p.NY, np2 = 2 * p.npml;
    if (yh.s >= 0) {
        float *psy = P + 6 * p.sx;
        const long long sy = p.sy;
        const int po = (k * np2 + yh.s) * pitch + i;
        float2 q0 = ld2(psy + hin * sy + po), q1 = ld2(psy + (hin + 1) * sy + po);
        rec2(q0, dEz_dy, yh.b, yh.a);
        rec2(q1, dEx_dy, yh.b, yh.a);
        if (wr) { st2(psy + hout * sy + po, q0); st2(psy + (hout + 1) * sy + po, q1); }
    }
    if (szh >= 0) {
        float *psz = P + 6 * p.sx + 6 * p.sy;
        const long long sz = p.sz;
        const int po = (szh * NY + j) * pitch + i;
        float2 q0 = ld2(psz + hin * sz + po), q1 = ld2(psz + (hin + 1) * sz + po);
        rec2(q0, dEy_dz, z.bzh, z.azh);
        rec2(q1, dEx_dz, z.bzh, z.azh);
        if (wr) { st2(psz + hout * sz + po, q0); st2(psz + (hout + 1) * sz + po, q1); }
    }
    if (xh.s0 >= 0 || xh.s1 >= 0) {
        float *psx = P;
        const long long sx = p.sx;
        const int ro = (k * NY + j) * np2;
        if (xh.s0 >= 0) {
            float q0 = psx[hin * sx + ro + xh.s0], q1 = psx[(hin + 1) * sx + ro + xh.s0];
            rec1(q0, dEz_dx.x, xh.b0, xh.a0);
            rec1(q1, dEy_dx.x, xh.b0, xh.a0);
            if (wr) { psx[hout * sx + ro + xh.s0] = q0; psx[(hout + 1) * sx + ro + xh.s0] = q1; }
        }
        if (xh.s1 >= 0) {
            float q0 = psx[hin * sx + ro + xh.s1], q1 = psx[(hin + 1) * sx + ro + xh.s1];
            rec1(q0, dEz_dx.y, xh.b1, xh.a1);
            rec1(q1, dEy_dx.y, xh.b1, xh.a1);
            if (wr) { psx[hout * sx + ro + xh.s1] = q0; psx[(hout + 1) * sx + ro + xh.s1] = q1; }
        }
    }
    const float cH = p.cH;
    hx = hupd(ld2(S0 + B3 + o), cH, dEz_dy, dEy_dz);
    hy = hupd(ld2(S0 + B3 + PL + o), cH, dEx_dz, dEz_dx);
    hz = hupd(ld2(S0 + B3 + 2 * PL + o), cH, dEy_dx, dEx_dy);
}

template <int BY, int MINB>
__global__ void __launch_bounds__(32 * (BY + 1), MINB)
    k_step_fz(const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmH,
              const __grid_constant__ CUtensorMap tmH2, const __grid_constant__ CUtensorMap tmQ,
              const StepParams<float> p, const int jstep, const int KZ, const int S) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[4];
    constexpr int RY = BY + 2, PL = RY * kXW, HPL = (BY + 1) * kXW;
    const int B3 = fz_block3(BY);
    const bool vti = p.qv != p.qh;
    const int nq = vti ? 2 : 1;
    const int stf = fz_stage_floats(BY, nq);
    constexpr int NST = fz_nst(BY, MINB);
    float *sm = reinterpret_cast<float *>(smem_raw);
    float *sHn = sm + NST * stf;                              // H^{n+1/2} of plane k: [3][BY+1][kXW]
    ZT *zt = reinterpret_cast<ZT *>(sHn + 3 * HPL);           // z tables of planes kstart .. k1
    const int tid = threadIdx.y * 32 + threadIdx.x;
    const int s = blockIdx.x % S;
    const int i0 = (blockIdx.x / S) * 64, j0 = blockIdx.y * BY;
    const bool halo = (threadIdx.y == BY);                   // the warp of row j0-1 and column i0-1
    const int i = i0 + 2 * threadIdx.x;
    const int j = halo ? j0 - 1 : j0 + threadIdx.y;
    const bool act = (i < p.nx) && (j >= 0) && (j < p.ny);
    const int k0 = blockIdx.z * KZ;
    const int k1 = min(k0 + KZ, p.nz);
    const int kstart = (k0 > 0) ? k0 - 1 : 0;
    const int n = *p.step + jstep;
    const int wE = (s * p.nslot + n % p.nslot) * 3;       // 4th coordinate of E^n's Ex in the ring map
    const CUtensorMap *mH = (n & 1) ? &tmH2 : &tmH;        // H^{n-1/2}
    const uint32_t bytes = (uint32_t)((6 + nq) * PL * sizeof(float));

    if (tid == 0) {
        for (int u = 0; u < NST; ++u) fz_bar_init(&bar[u]);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int u = tid; u < 3 * HPL; u += 32 * (BY + 1)) sHn[u] = 0.f;   // faces nobody computes stay zero
    for (int m = kstart + tid; m <= k1; m += 32 * (BY + 1)) {
        ZT z;
        z.ihzh = __ldg(p.lz.ih_h + m); z.ihzn = __ldg(p.lz.ih_n + m);
        z.bzh = __ldg(p.lz.b_h + m); z.azh = __ldg(p.lz.a_h + m);
        z.bzn = __ldg(p.lz.b_n + m); z.azn = __ldg(p.lz.a_n + m);
        z.gzh = __ldg(p.gz.h + m); z.gzs = __ldg(p.gz.s + m);
        z.szh = slab_half(m, p.nz, p.npml); z.szn = slab_node(m, p.nz, p.npml);
        z.pad0 = z.pad1 = 0;
        zt[m - kstart] = z;
    }
    __syncthreads();
    // plane m lives in stage (m - kstart) % NST; the stage and parity bookkeeping below
    // advances incrementally (no integer division in the plane loop)
    auto issue = [&](int m, int u) {
        float *d = sm + u * stf;
        fz_expect(&bar[u], bytes + (m == kstart ? (uint32_t)p.fault_tx : 0u));
        fz_tile4(d, &tmE, i0 - 4, j0 - 1, m, wE, &bar[u]);
        fz_tile4(d + B3, mH, i0 - 4, j0 - 1, m, s * 3, &bar[u]);
        fz_tile4(d + 2 * B3, &tmQ, i0 - 4, j0 - 1, m, 0, &bar[u]);
    };
    if (tid == 0)
        for (int m = kstart; m <= min(kstart + NST - 2, k1); ++m) issue(m, m - kstart);
    int inext = kstart + NST - 1;                          // next plane to issue, into stage ist
    int ist = NST - 1;

    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch, NY = p.NY;
    const int nx = p.nx, ny = p.ny, npml = p.npml, np2 = 2 * npml;
    const long long sb = (long long)s * p.ering_stride;
    float *__restrict__ En = p.ering + sb + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    float *__restrict__ Ho = ((n & 1) ? p.H : p.H2) + (long long)s * 3 * p.vol;
    float *P = p.psi + (long long)s * p.psi_stride;
    const int hin = (n & 1) ? 4 : 0, hout = 4 - hin;
    float *psx = P, *psy = P + 6 * p.sx, *psz = P + 6 * p.sx + 6 * p.sy;
    const long long sx = p.sx, sy = p.sy, sz = p.sz;
    const float K2 = p.k2w0dt;

    // per-thread constants (in-range entries for threads off the lattice)
    const int ic = act ? i : 0, jc = act ? j : 0;
    const XH xh = xh_of(p, ic);
    const YH yh = yh_of(p, jc);
    const float2 ihxn = ld2(p.lx.ih_n + ic), gxh = ld2(p.gx.h + ic), gxs = ld2(p.gx.s + ic);
    const int sxn0 = slab_node(ic, nx, npml), sxn1 = slab_node(ic + 1, nx, npml);
    const float ihyn = __ldg(p.ly.ih_n + jc), byn = __ldg(p.ly.b_n + jc), ayn = __ldg(p.ly.a_n + jc);
    const int syn = slab_node(jc, ny, npml);
    const float gyh = __ldg(p.gy.h + jc), gys = __ldg(p.gy.s + jc);
    const bool taps = act && !halo && p.colmap && p.inc && p.tflag[s * p.tflag_stride + jc * p.nseg + (ic >> 5)];
    const int r = halo ? 0 : threadIdx.y + 1;                  // staged row of the thread's cells
    const int o = r * kXW + 2 * threadIdx.x + 4;                // staged offset of cell i
    // the halo warp's column task: lane l < BY computes Hy, Hz at (i0-1, j0+l)
    const int cj = j0 + threadIdx.x;
    const bool col = halo && threadIdx.x < BY && i0 > 0 && cj < ny;
    const int co = (threadIdx.x + 1) * kXW + 3;

    float2 hxm = f2(0.f, 0.f), hym = f2(0.f, 0.f);       // own Hx, Hy of H^{n+1/2}, plane k-1
    float2 Aq = f2(0.f, 0.f), Bq = f2(0.f, 0.f);         // plane k-1 cell sums of the Ex / Ey edges
    int k = kstart;
    int st0 = 0;                                           // stage of plane k
    uint32_t ph = 1;                                       // bit u: parity of stage u's next completion
    bool ok = mbar_wait_bounded(&bar[0], 0);
    for (; k < k1; ++k) {
        const int st1 = (st0 + 1 == NST) ? 0 : st0 + 1;    // stage of plane k+1
        if (ok) ok = mbar_wait_bounded(&bar[st1], (ph >> st1) & 1u);
        ph ^= 1u << st1;
        // every thread has its planes and the stage of plane k-1 and sHn are free; a
        // give-up anywhere ends the loop for the whole block
        if (__syncthreads_or(!ok)) break;
        if (inext <= k1) {
            if (tid == 0) issue(inext, ist);
            ++inext;
            ist = (ist + 1 == NST) ? 0 : ist + 1;
        }
        const bool own = (k >= k0);
        const float *S0 = sm + st0 * stf, *S1 = sm + st1 * stf;
        st0 = st1;
        const ZT z = zt[k - kstart];
        const int szh = z.szh;
        // ---- phase 1: H^{n+1/2} of the tile (own rows), of row j0-1 and column i0-1 (halo warp)
        float2 hxn = f2(0.f, 0.f), hyn = hxn, hzn = hxn;
        if (act) {
            h_pair(p, S0, S1, B3, PL, o, i, j, k, szh, z, xh, yh, own && !halo, P, hin, hout, hxn, hyn, hzn);
            st2(sHn + o, hxn);
            st2(sHn + HPL + o, hyn);
            st2(sHn + 2 * HPL + o, hzn);
        }
        if (col) {                     // Hy, Hz at (i0-1, cj): CPML memory read only
            const int ci = i0 - 1;
            const float *Ex0 = S0, *Ey0 = S0 + PL, *Ez0 = S0 + 2 * PL;
            const float ihx = __ldg(p.lx.ih_h + ci), ihy = __ldg(p.ly.ih_h + cj);
            float d_xz = (S1[co] - Ex0[co]) * z.ihzh, d_zx = (Ez0[co + 1] - Ez0[co]) * ihx;
            float d_yx = (Ey0[co + 1] - Ey0[co]) * ihx, d_xy = (Ex0[co + kXW] - Ex0[co]) * ihy;
            const int sxh = slab_half(ci, nx, npml), syh = slab_half(cj, ny, npml);
            if (szh >= 0) d_xz += z.bzh * psz[(hin + 1) * sz + (szh * NY + cj) * pitch + ci] + z.azh * d_xz;
            if (sxh >= 0) {
                const float b = __ldg(p.lx.b_h + ci), a = __ldg(p.lx.a_h + ci);
                const int po = (k * NY + cj) * np2 + sxh;
                d_zx += b * psx[hin * sx + po] + a * d_zx;
                d_yx += b * psx[(hin + 1) * sx + po] + a * d_yx;
            }
            if (syh >= 0) {
                const float b = __ldg(p.ly.b_h + cj), a = __ldg(p.ly.a_h + cj);
                d_xy += b * psy[(hin + 1) * sy + (k * np2 + syh) * pitch + ci] + a * d_xy;
            }
            sHn[HPL + co] = S0[B3 + PL + co] - p.cH * (d_xz - d_zx);
            sHn[2 * HPL + co] = S0[B3 + 2 * PL + co] - p.cH * (d_yx - d_xy);
        }
        __syncthreads();
        if (!act || halo) continue;
        const float *Q0 = S0 + 2 * B3;
        const float2 qc = ld2(Q0 + o), qD = ld2(Q0 + o - kXW);
        const float qL = Q0[o - 1];
        const float2 Ak = f2(qD.x + qc.x, qD.y + qc.y);     // cells j-1, j of the Ex edges
        const float2 Bk = f2(qL + qc.x, qc.x + qc.y);        // cells i-1, i of the Ey edges
        if (!own) {                                           // plane k0-1: only Hx, Hy are needed
            hxm = hxn; hym = hyn; Aq = Ak; Bq = Bk;
            continue;
        }
        const int idx = k * plane + j * pitch + i;
        st2(Ho + idx, hxn);
        st2(Ho + vol + idx, hyn);
        st2(Ho + 2 * vol + idx, hzn);

        // ---- phase 2: E^{n+1} on the thread's cells, neighbours of H from shared memory
        const float2 ex = ld2(S0 + o), ey = ld2(S0 + PL + o), ez = ld2(S0 + 2 * PL + o);
        const float hzL = sHn[2 * HPL + o - 1], hyL = sHn[HPL + o - 1];
        const float2 hzD = ld2(sHn + 2 * HPL + o - kXW), hxD = ld2(sHn + o - kXW);
        float2 dHz_dy = dsc(hzn, hzD, ihyn), dHy_dz = dsc(hyn, hym, z.ihzn);
        float2 dHx_dz = dsc(hxn, hxm, z.ihzn), dHz_dx = dsc(hzn, f2(hzL, hzn.x), ihxn);
        float2 dHy_dx = dsc(hyn, f2(hyL, hyn.x), ihxn), dHx_dy = dsc(hxn, hxD, ihyn);
        if (syn >= 0) {
            const int po = (k * np2 + syn) * pitch + i;
            float2 q2 = ld2(psy + 2 * sy + po), q3 = ld2(psy + 3 * sy + po);
            rec2(q2, dHz_dy, byn, ayn);
            rec2(q3, dHx_dy, byn, ayn);
            st2(psy + 2 * sy + po, q2);
            st2(psy + 3 * sy + po, q3);
        }
        const int szn = z.szn;
        if (szn >= 0) {
            const int po = (szn * NY + j) * pitch + i;
            float2 q2 = ld2(psz + 2 * sz + po), q3 = ld2(psz + 3 * sz + po);
            rec2(q2, dHy_dz, z.bzn, z.azn);
            rec2(q3, dHx_dz, z.bzn, z.azn);
            st2(psz + 2 * sz + po, q2);
            st2(psz + 3 * sz + po, q3);
        }
        if (sxn0 >= 0 || sxn1 >= 0) {
            const int ro = (k * NY + j) * np2;
            if (sxn0 >= 0) {
                const float b = __ldg(p.lx.b_n + i), a = __ldg(p.lx.a_n + i);
                float q2 = psx[2 * sx + ro + sxn0], q3 = psx[3 * sx + ro + sxn0];
                rec1(q2, dHz_dx.x, b, a);
                rec1(q3, dHy_dx.x, b, a);
                psx[2 * sx + ro + sxn0] = q2;
                psx[3 * sx + ro + sxn0] = q3;
            }
            if (sxn1 >= 0) {
                const float b = __ldg(p.lx.b_n + i + 1), a = __ldg(p.lx.a_n + i + 1);
                float q2 = psx[2 * sx + ro + sxn1], q3 = psx[3 * sx + ro + sxn1];
                rec1(q2, dHz_dx.y, b, a);
                rec1(q3, dHy_dx.y, b, a);
                psx[2 * sx + ro + sxn1] = q2;
                psx[3 * sx + ro + sxn1] = q3;
            }
        }
        // dt/eps of the three edges from the cell values (zero on the PEC edges)
        const float *Qz = Q0 + (nq - 1) * PL;             // sigma_v of a VTI medium, else sigma
        const float2 vc = ld2(Qz + o), vD = ld2(Qz + o - kXW);
        const float vL = Qz[o - 1], vDL = Qz[o - 1 - kXW];
        const float2 Cz = f2(vL + vc.x, vc.x + vc.y), Dz = f2(vDL + vD.x, vD.x + vD.y);
        const bool jk = (j > 0) && (k > 0);
        const float kxz = K2 * gys * z.gzs, kyz = K2 * gyh * z.gzs, kzz = K2 * gys * z.gzh;
        const float cx0 = jk ? __fdividef(kxz * gxh.x, Aq.x + Ak.x) : 0.f;
        const float cx1 = jk ? __fdividef(kxz * gxh.y, Aq.y + Ak.y) : 0.f;
        const float cy0 = (i > 0 && k > 0) ? __fdividef(kyz * gxs.x, Bq.x + Bk.x) : 0.f;
        const float cy1 = (k > 0) ? __fdividef(kyz * gxs.y, Bq.y + Bk.y) : 0.f;
        const float cz0 = (i > 0 && j > 0) ? __fdividef(kzz * gxs.x, Cz.x + Dz.x) : 0.f;
        const float cz1 = (j > 0) ? __fdividef(kzz * gxs.y, Cz.y + Dz.y) : 0.f;
        float2 exn = f2(ex.x + cx0 * (dHz_dy.x - dHy_dz.x), ex.y + cx1 * (dHz_dy.y - dHy_dz.y));
        float2 eyn = f2(ey.x + cy0 * (dHx_dz.x - dHz_dx.x), ey.y + cy1 * (dHx_dz.y - dHz_dx.y));
        float2 ezn = f2(ez.x + cz0 * (dHy_dx.x - dHx_dy.x), ez.y + cz1 * (dHy_dx.y - dHx_dy.y));
        if (taps) {
            const int2 *cm = p.colmap + (long long)s * p.colmap_stride + j * pitch + i;
            const int *tk = p.tapk + (long long)s * p.itap_stride;
            const float *inc = p.inc + ((long long)jstep * S + s) * p.inc_ntl;
            const int2 c0 = __ldg(cm), c1 = __ldg(cm + 1);
            if (c0.y) { const float3 a = taps_at(tk, inc, k, c0); exn.x += a.x; eyn.x += a.y; ezn.x += a.z; }
            if (c1.y) { const float3 a = taps_at(tk, inc, k, c1); exn.y += a.x; eyn.y += a.y; ezn.y += a.z; }
        }
        st2(En + idx, exn);
        st2(En + vol + idx, eyn);
        st2(En + 2 * vol + idx, ezn);
        hxm = hxn; hym = hyn; Aq = Ak; Bq = Bk;
    }
    if (k < k1) {                      // gave up on a stage: report, let the issued copies land
        if (tid == 0) {
            atomicOr(p.err, kErrOnepassWait);
            for (int m = k; m < inext; ++m)
                mbar_wait_bounded(&bar[(m - kstart) % NST], (uint32_t)(((m - kstart) / NST) & 1));
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Warp-specialised fused step (Sec. 2, Eq. 4 with the unsplit CPML): the H
// half-step and the E step of one step in one kernel, each field read from DRAM
// once, with the two halves on different warps.
//
// A block owns 64 cells (x) by BY rows (y) and marches a z block of KZ planes;
// every thread of a row warp owns two consecutive cells (i, i+1).  Its warps:
//  * BY + 1 producer warps: H^{n+1/2} of rows j0-1 .. j0+BY-1 from E^n and
//    H^{n-1/2} in global memory (L1/L2 serve the neighbours), written to a
//    shared plane buffer and, for the block's own rows and planes, to the other
//    H buffer in global memory.  Row j0-1 belongs to the block below in y: it is
//    recomputed here, not exchanged, so no block waits on another; H and the CPML
//    memory of the H update are therefore double buffered (step n reads the
//    buffer of parity n, writes the other), as for k_step_fz;
//  * one column warp: Hy and Hz of column i0-1 (lane l: row j0+l), recomputed
//    the same way;
//  * BY consumer warps: E^{n+1} of rows j0 .. j0+BY-1 from E^n (just read by the
//    producers: an L1 hit), dt/eps with the PEC edges zeroed, H^{n+1/2} of the
//    plane from the shared buffer (i-1 and j-1 neighbours included) and of plane
//    k-1 from registers; the CPML memory of the E update in place (one owner).
// The producers fill one of two plane buffers while the consumers drain the
// other: per buffer a "full" mbarrier (every producer thread arrives) and an
// "empty" mbarrier (every consumer thread arrives after reading, only when the
// producers will refill it), every wait bounded (about a second); a thread that
// gives up raises the one-pass bit of *err and leaves its loop, so the others'
// waits run out too and the kernel returns (the copy-fault test hook makes the
// producers skip their first arrival).  A z block starting at k0 > 0 first
// produces plane k0-1 (not stored) for the consumers' k-1 values.  blockIdx.x
// runs over (x tile, source) with the source fastest.
// ---------------------------------------------------------------------------
namespace {
constexpr int kWsW = 68;           // shared row: column c holds cell i0 - 2 + c (i0-1 at 1, i0 at 2)

__device__ __forceinline__ void ws_bar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void ws_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s_u32(b)) : "memory");
}
}  // namespace

// Inputs of one producer plane k at the thread's cells: E^n (Ez at k, Ex and Ey at k+1, the i+2
// and j+1 neighbours) and H^{n-1/2}, all loaded before any is used.
struct WsIn {
    float2 ez, exk, eyk, exU, ezU, hx, hy, hz;
    float ezR, eyR;
};
__device__ __forceinline__ WsIn ws_load(const float *__restrict__ E, const float *__restrict__ Hi, int idx, int vol,
                                        int plane, int pitch) {
    WsIn a;
    a.ez = ld2(E + 2 * vol + idx);
    a.exk = ld2(E + idx + plane); a.eyk = ld2(E + vol + idx + plane);
    a.ezR = __ldg(E + 2 * vol + idx + 2); a.eyR = __ldg(E + vol + idx + 2);
    a.exU = ld2(E + idx + pitch); a.ezU = ld2(E + 2 * vol + idx + pitch);
    a.hx = ld2(Hi + idx); a.hy = ld2(Hi + vol + idx); a.hz = ld2(Hi + 2 * vol + idx);
    return a;
}

template <int BY, int MINB>
__global__ void __launch_bounds__(32 * (2 * BY + 2), MINB)
    k_step_ws(const StepParams<float> p, const int jstep, const int KZ, const int S) {
    constexpr int NB = 2, RW = BY + 1, PLF = 3 * RW * kWsW;
    __shared__ __align__(16) float sH[NB * PLF];
    __shared__ __align__(8) uint64_t full[NB], empty[NB];
    const int w = threadIdx.y, lane = threadIdx.x;
    const int tid = w * 32 + lane;
    const int s = blockIdx.x % S;
    const int i0 = (blockIdx.x / S) * 64, j0 = blockIdx.y * BY;
    const int i = i0 + 2 * lane;
    const int k0 = blockIdx.z * KZ;
    const int k1 = min(k0 + KZ, p.nz);
    const int kstart = (k0 > 0) ? k0 - 1 : 0;
    const int T = k1 - kstart;                     // planes produced (the first is k0-1 when k0 > 0)
    constexpr int NPROD = 32 * (BY + 2), NCONS = 32 * BY;
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            ws_bar_init(&full[b], NPROD);
            ws_bar_init(&empty[b], NCONS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int u = tid; u < NB * PLF; u += 32 * (2 * BY + 2)) sH[u] = 0.f;   // cells nobody computes stay zero
    __syncthreads();

    const int n = *p.step + jstep;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch, NY = p.NY;
    const int nx = p.nx, ny = p.ny, npml = p.npml, np2 = 2 * npml;
    const long long sb = (long long)s * p.ering_stride;
    const float *__restrict__ E = p.ering + sb + (long long)(n % p.nslot) * 3 * p.vol;      // E^n
    const int hin = (n & 1) ? 4 : 0, hout = 4 - hin;
    float *P = p.psi + (long long)s * p.psi_stride;
    float *psx = P, *psy = P + 6 * p.sx, *psz = P + 6 * p.sx + 6 * p.sy;
    const long long sx = p.sx, sy = p.sy, sz = p.sz;
    const float cH = p.cH;
    bool ok = true;

    if (w <= BY) {
        // ---- producer: H^{n+1/2} of row j0-1+w
        const float *__restrict__ Hi = ((n & 1) ? p.H2 : p.H) + (long long)s * 3 * vol;
        float *__restrict__ Ho = ((n & 1) ? p.H : p.H2) + (long long)s * 3 * vol;
        const int j = j0 - 1 + w;
        const bool act = (i < nx) && (j >= 0) && (j < ny);
        const bool own = (w >= 1);
        const int ic = act ? i : 0, jc = act ? j : 0;
        const XH xh = xh_of(p, ic);
        const YH yh = yh_of(p, jc);
        const int o = w * kWsW + 2 + 2 * lane;     // shared offset of cell i in row w
        int idx = kstart * plane + jc * pitch + ic;
        float2 ex = act ? ld2(E + idx) : f2(0.f, 0.f), ey = act ? ld2(E + vol + idx) : f2(0.f, 0.f);
        for (int t = 0; t < T; ++t, idx += plane) {
            const int k = kstart + t, b = t & 1;
            // H^{n+1/2} of the plane in registers first (its loads need no buffer), then the wait
            // for the buffer, so the wait overlaps the loads
            float2 hx = f2(0.f, 0.f), hy = hx, hz = hx;
            if (act) {
                const WsIn cur = ws_load(E, Hi, idx, vol, plane, pitch);   // every load of the plane first
                const float2 ez = cur.ez, exk = cur.exk, eyk = cur.eyk, exU = cur.exU, ezU = cur.ezU;
                const float ezR = cur.ezR, eyR = cur.eyR;
                const float ihz = __ldg(p.lz.ih_h + k);
                float2 dEz_dy = dsc(ezU, ez, yh.ih), dEx_dy = dsc(exU, ex, yh.ih);
                float2 dEy_dz = dsc(eyk, ey, ihz), dEx_dz = dsc(exk, ex, ihz);
                float2 dEz_dx = dsc(f2(ez.y, ezR), ez, xh.ih), dEy_dx = dsc(f2(ey.y, eyR), ey, xh.ih);
                const bool wr = own && (k >= k0);
                if (yh.s >= 0) {
                    const int po = (k * np2 + yh.s) * pitch + i;
                    float2 q0 = ld2(psy + hin * sy + po), q1 = ld2(psy + (hin + 1) * sy + po);
                    rec2(q0, dEz_dy, yh.b, yh.a);
                    rec2(q1, dEx_dy, yh.b, yh.a);
                    if (wr) { st2(psy + hout * sy + po, q0); st2(psy + (hout + 1) * sy + po, q1); }
                }
                const int szh = slab_half(k, p.nz, npml);
                if (szh >= 0) {
                    const float bz = __ldg(p.lz.b_h + k), az = __ldg(p.lz.a_h + k);
                    const int po = (szh * NY + j) * pitch + i;
                    float2 q0 = ld2(psz + hin * sz + po), q1 = ld2(psz + (hin + 1) * sz + po);
                    rec2(q0, dEy_dz, bz, az);
                    rec2(q1, dEx_dz, bz, az);
                    if (wr) { st2(psz + hout * sz + po, q0); st2(psz + (hout + 1) * sz + po, q1); }
                }
                if (xh.s0 >= 0 || xh.s1 >= 0) {
                    const int ro = (k * NY + j) * np2;
                    if (xh.s0 >= 0) {
                        float q0 = psx[hin * sx + ro + xh.s0], q1 = psx[(hin + 1) * sx + ro + xh.s0];
                        rec1(q0, dEz_dx.x, xh.b0, xh.a0);
                        rec1(q1, dEy_dx.x, xh.b0, xh.a0);
                        if (wr) { psx[hout * sx + ro + xh.s0] = q0; psx[(hout + 1) * sx + ro + xh.s0] = q1; }
                    }
                    if (xh.s1 >= 0) {
                        float q0 = psx[hin * sx + ro + xh.s1], q1 = psx[(hin + 1) * sx + ro + xh.s1];
                        rec1(q0, dEz_dx.y, xh.b1, xh.a1);
                        rec1(q1, dEy_dx.y, xh.b1, xh.a1);
                        if (wr) { psx[hout * sx + ro + xh.s1] = q0; psx[(hout + 1) * sx + ro + xh.s1] = q1; }
                    }
                }
                hx = hupd(cur.hx, cH, dEz_dy, dEy_dz);
                hy = hupd(cur.hy, cH, dEx_dz, dEz_dx);
                hz = hupd(cur.hz, cH, dEy_dx, dEx_dy);
                if (wr) {
                    st2(Ho + idx, hx);
                    st2(Ho + vol + idx, hy);
                    st2(Ho + 2 * vol + idx, hz);
                }
                ex = exk;
                ey = eyk;
            }
            if (t >= NB && ok) ok = mbar_wait_bounded(&empty[b], (uint32_t)((t / NB - 1) & 1));
            if (!ok) break;
            if (act) {
                float *sb_ = sH + b * PLF;
                st2(sb_ + o, hx);
                st2(sb_ + RW * kWsW + o, hy);
                st2(sb_ + 2 * RW * kWsW + o, hz);
            }
            if (!(t == 0 && p.fault_tx)) ws_arrive(&full[b]);   // test hook: the first arrival never comes
        }
    } else if (w == BY + 1) {
        // ---- column warp: Hy, Hz of cell i0-1 in row j0+lane (CPML memory read only)
        const float *__restrict__ Hi = ((n & 1) ? p.H2 : p.H) + (long long)s * 3 * vol;
        const int ci = i0 - 1, cj = j0 + lane;
        const bool act = (lane < BY) && (i0 > 0) && (cj < ny);
        const int cic = act ? ci : 0, cjc = act ? cj : 0;
        const float ihx = __ldg(p.lx.ih_h + cic), ihy = __ldg(p.ly.ih_h + cjc);
        const int sxh = slab_half(cic, nx, npml), syh = slab_half(cjc, ny, npml);
        const float bx = act && sxh >= 0 ? __ldg(p.lx.b_h + cic) : 0.f, ax = act && sxh >= 0 ? __ldg(p.lx.a_h + cic) : 0.f;
        const float by = act && syh >= 0 ? __ldg(p.ly.b_h + cjc) : 0.f, ay = act && syh >= 0 ? __ldg(p.ly.a_h + cjc) : 0.f;
        const int co = (1 + lane) * kWsW + 1;
        int idx = kstart * plane + cjc * pitch + cic;
        for (int t = 0; t < T; ++t, idx += plane) {
            const int k = kstart + t, b = t & 1;
            float hy = 0.f, hz = 0.f;
            if (act) {
                const float ihz = __ldg(p.lz.ih_h + k);
                const float exc = __ldg(E + idx);
                float d_xz = (__ldg(E + idx + plane) - exc) * ihz;
                float d_zx = (__ldg(E + 2 * vol + idx + 1) - __ldg(E + 2 * vol + idx)) * ihx;
                float d_yx = (__ldg(E + vol + idx + 1) - __ldg(E + vol + idx)) * ihx;
                float d_xy = (__ldg(E + idx + pitch) - exc) * ihy;
                const int szh = slab_half(k, p.nz, npml);
                if (szh >= 0) {
                    const float bz = __ldg(p.lz.b_h + k), az = __ldg(p.lz.a_h + k);
                    d_xz += bz * psz[(hin + 1) * sz + (szh * NY + cj) * pitch + ci] + az * d_xz;
                }
                if (sxh >= 0) {
                    const int po = (k * NY + cj) * np2 + sxh;
                    d_zx += bx * psx[hin * sx + po] + ax * d_zx;
                    d_yx += bx * psx[(hin + 1) * sx + po] + ax * d_yx;
                }
                if (syh >= 0) d_xy += by * psy[(hin + 1) * sy + (k * np2 + syh) * pitch + ci] + ay * d_xy;
                hy = __ldg(Hi + vol + idx) - cH * (d_xz - d_zx);
                hz = __ldg(Hi + 2 * vol + idx) - cH * (d_yx - d_xy);
            }
            if (t >= NB && ok) ok = mbar_wait_bounded(&empty[b], (uint32_t)((t / NB - 1) & 1));
            if (!ok) break;
            if (act) {
                float *sb_ = sH + b * PLF;
                sb_[RW * kWsW + co] = hy;
                sb_[2 * RW * kWsW + co] = hz;
            }
            if (!(t == 0 && p.fault_tx)) ws_arrive(&full[b]);   // test hook: the first arrival never comes
        }
    } else {
        // ---- consumer: E^{n+1} of row j0 + r - 1
        const int r = w - BY - 1;                  // shared row of the thread's cells (1 .. BY)
        const int j = j0 + r - 1;
        const bool act = (i < nx) && (j < ny);
        const int ic = act ? i : 0, jc = act ? j : 0;
        float *__restrict__ En = p.ering + sb + (long long)((n + 1) % p.nslot) * 3 * p.vol;
        const float2 ihxn = ld2(p.lx.ih_n + ic);
        const int sxn0 = slab_node(ic, nx, npml), sxn1 = slab_node(ic + 1, nx, npml);
        const float ihyn = __ldg(p.ly.ih_n + jc), byn = __ldg(p.ly.b_n + jc), ayn = __ldg(p.ly.a_n + jc);
        const int syn = slab_node(jc, ny, npml);
        const bool taps = act && p.colmap && p.inc && p.tflag[s * p.tflag_stride + jc * p.nseg + (ic >> 5)];
        const float *__restrict__ cE = p.cEm;
        const int o = r * kWsW + 2 + 2 * lane;
        float2 hxm = f2(0.f, 0.f), hym = f2(0.f, 0.f);   // H^{n+1/2} of plane k-1 at the thread's cells
        int idx = kstart * plane + jc * pitch + ic;
        for (int t = 0; t < T; ++t, idx += plane) {
            const int k = kstart + t, b = t & 1;
            const bool upd = act && (k >= k0);
            // the values that do not depend on the plane's H first, so their loads overlap the wait
            float2 ex = f2(0.f, 0.f), ey = ex, ez = ex, c0 = ex, c1 = ex, c2 = ex;
            if (upd) {
                ex = ld2(E + idx); ey = ld2(E + vol + idx); ez = ld2(E + 2 * vol + idx);
                c0 = ld2(cE + idx); c1 = ld2(cE + vol + idx); c2 = ld2(cE + 2 * vol + idx);
            }
            if (ok) ok = mbar_wait_bounded(&full[b], (uint32_t)((t / NB) & 1));
            if (!ok) break;
            const float *sb_ = sH + b * PLF;
            const float *SX = sb_, *SY = sb_ + RW * kWsW, *SZ = sb_ + 2 * RW * kWsW;
            const float2 hxn = ld2(SX + o), hyn = ld2(SY + o), hzn = ld2(SZ + o);
            const float hzL = SZ[o - 1], hyL = SY[o - 1];
            const float2 hzD = ld2(SZ + o - kWsW), hxD = ld2(SX + o - kWsW);
            if (t + NB < T) ws_arrive(&empty[b]);
            if (!upd) {                            // plane k0-1: only its H is needed
                hxm = hxn; hym = hyn;
                continue;
            }
            const float ihz = __ldg(p.lz.ih_n + k);
            float2 dHz_dy = dsc(hzn, hzD, ihyn), dHy_dz = dsc(hyn, hym, ihz);
            float2 dHx_dz = dsc(hxn, hxm, ihz), dHz_dx = dsc(hzn, f2(hzL, hzn.x), ihxn);
            float2 dHy_dx = dsc(hyn, f2(hyL, hyn.x), ihxn), dHx_dy = dsc(hxn, hxD, ihyn);
            if (syn >= 0) {
                const int po = (k * np2 + syn) * pitch + i;
                float2 q2 = ld2(psy + 2 * sy + po), q3 = ld2(psy + 3 * sy + po);
                rec2(q2, dHz_dy, byn, ayn);
                rec2(q3, dHx_dy, byn, ayn);
                st2(psy + 2 * sy + po, q2);
                st2(psy + 3 * sy + po, q3);
            }
            const int szn = slab_node(k, p.nz, npml);
            if (szn >= 0) {
                const float bz = __ldg(p.lz.b_n + k), az = __ldg(p.lz.a_n + k);
                const int po = (szn * NY + j) * pitch + i;
                float2 q2 = ld2(psz + 2 * sz + po), q3 = ld2(psz + 3 * sz + po);
                rec2(q2, dHy_dz, bz, az);
                rec2(q3, dHx_dz, bz, az);
                st2(psz + 2 * sz + po, q2);
                st2(psz + 3 * sz + po, q3);
            }
            if (sxn0 >= 0 || sxn1 >= 0) {
                const int ro = (k * NY + j) * np2;
                if (sxn0 >= 0) {
                    const float bb = __ldg(p.lx.b_n + i), aa = __ldg(p.lx.a_n + i);
                    float q2 = psx[2 * sx + ro + sxn0], q3 = psx[3 * sx + ro + sxn0];
                    rec1(q2, dHz_dx.x, bb, aa);
                    rec1(q3, dHy_dx.x, bb, aa);
                    psx[2 * sx + ro + sxn0] = q2;
                    psx[3 * sx + ro + sxn0] = q3;
                }
                if (sxn1 >= 0) {
                    const float bb = __ldg(p.lx.b_n + i + 1), aa = __ldg(p.lx.a_n + i + 1);
                    float q2 = psx[2 * sx + ro + sxn1], q3 = psx[3 * sx + ro + sxn1];
                    rec1(q2, dHz_dx.y, bb, aa);
                    rec1(q3, dHy_dx.y, bb, aa);
                    psx[2 * sx + ro + sxn1] = q2;
                    psx[3 * sx + ro + sxn1] = q3;
                }
            }
            float2 exn = f2(ex.x + c0.x * (dHz_dy.x - dHy_dz.x), ex.y + c0.y * (dHz_dy.y - dHy_dz.y));
            float2 eyn = f2(ey.x + c1.x * (dHx_dz.x - dHz_dx.x), ey.y + c1.y * (dHx_dz.y - dHz_dx.y));
            float2 ezn = f2(ez.x + c2.x * (dHy_dx.x - dHx_dy.x), ez.y + c2.y * (dHy_dx.y - dHx_dy.y));
            if (taps) {
                const int2 *cm = p.colmap + (long long)s * p.colmap_stride + j * pitch + i;
                const int *tk = p.tapk + (long long)s * p.itap_stride;
                const float *inc = p.inc + ((long long)jstep * S + s) * p.inc_ntl;
                const int2 m0 = __ldg(cm), m1 = __ldg(cm + 1);
                if (m0.y) { const float3 a = taps_at(tk, inc, k, m0); exn.x += a.x; eyn.x += a.y; ezn.x += a.z; }
                if (m1.y) { const float3 a = taps_at(tk, inc, k, m1); exn.y += a.x; eyn.y += a.y; ezn.y += a.z; }
            }
            st2(En + idx, exn);
            st2(En + vol + idx, eyn);
            st2(En + 2 * vol + idx, ezn);
            hxm = hxn; hym = hyn;
        }
    }
    if (!ok) atomicOr(p.err, kErrOnepassWait);
}

// V sigma of every cell on the lattice (zero off the cells), sigma_h into qh and,
// for a VTI medium, sigma_v into qv: the per-cell material value of k_step_fz.
__global__ void k_qcell(const GeoD g, const float *__restrict__ rho, const float *__restrict__ rho_z,
                        float *__restrict__ qh, float *__restrict__ qv) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.vol) return;
    const int i = (int)(t % g.pitch);
    const long long r = t / g.pitch;
    const int j = (int)(r % g.NY);
    const int k = (int)(r / g.NY);
    float a = 0.f, b = 0.f;
    if (i < g.nx && j < g.ny && k < g.nz) {
        const double V = g.hx[i] * g.hy[j] * g.hz[k];
        const long long c = ((long long)k * g.ny + j) * g.nx + i;
        const double rh = (double)rho[c];
        if (rh > 0.0 && isfinite(rh)) a = (float)(V / rh);
        if (qv) {
            const double rz = (double)rho_z[c];
            if (rz > 0.0 && isfinite(rz)) b = (float)(V / rz);
        }
    }
    qh[t] = a;
    if (qv) qv[t] = b;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mu;

// 4-D map of a stack of lattice volumes [w][NZ][NY][pitch] (FP32), box kXW x (by+2) x 1 x bw
cudaError_t encode_vol(CUtensorMap *m, const float *base, const StepParams<float> &p, long long w, int by, int bw) {
    {
        std::lock_guard<std::mutex> lk(g_encode_mu);
        if (!g_encode) {
            cudaDriverEntryPointQueryResult q;
            void *fn = nullptr;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fn)
                return cudaErrorNotSupported;
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        }
    }
    const cuuint64_t dims[4] = {(cuuint64_t)p.pitch, (cuuint64_t)p.NY, (cuuint64_t)p.NZ, (cuuint64_t)w};
    const cuuint64_t strides[3] = {(cuuint64_t)p.pitch * 4, (cuuint64_t)p.plane * 4, (cuuint64_t)p.vol * 4};
    const cuuint32_t box[4] = {(cuuint32_t)kXW, (cuuint32_t)(by + 2), 1, (cuuint32_t)bw};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box, es,
                                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}


template <int BY, int MB>
cudaError_t go_fz(const StepParams<float> &p, int S, int jstep, cudaStream_t st) {
    const int nq = (p.qv != p.qh) ? 2 : 1;
    constexpr int nst = fz_nst(BY, MB);
    const size_t smem = ((size_t)nst * fz_stage_floats(BY, nq) + 3 * (BY + 1) * kXW) * sizeof(float) +
                        (size_t)(p.FZ_kz + 2) * sizeof(ZT);
    static size_t set_smem[64] = {};               // per device: largest dynamic size configured so far
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (smem > set_smem[dev]) {
        cudaError_t e = cudaFuncSetAttribute(k_step_fz<BY, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_smem[dev] = smem;
    }
    CUtensorMap mE, mH, mH2, mQ;
    cudaError_t e = encode_vol(&mE, p.ering, p, (long long)S * p.nslot * 3, BY, 3);
    if (e == cudaSuccess) e = encode_vol(&mH, p.H, p, (long long)S * 3, BY, 3);
    if (e == cudaSuccess) e = encode_vol(&mH2, p.H2, p, (long long)S * 3, BY, 3);
    if (e == cudaSuccess) e = encode_vol(&mQ, p.qh, p, nq, BY, nq);
    if (e != cudaSuccess) return e;
    const int kz = p.FZ_kz;
    const dim3 grid((unsigned)(((p.nx / 2 + 31) / 32) * S), (unsigned)((p.ny + BY - 1) / BY),
                    (unsigned)((p.nz + kz - 1) / kz));
    k_step_fz<BY, MB><<<grid, dim3(32, BY + 1), smem, st>>>(mE, mH, mH2, mQ, p, jstep, kz, S);
    return cudaSuccess;
}
}  // namespace

template <int BY, int MB>
void go_ws(const StepParams<float> &p, int S, int jstep, cudaStream_t st) {
    const int kz = p.FZ_kz;
    const dim3 grid((unsigned)(((p.nx / 2 + 31) / 32) * S), (unsigned)((p.ny + BY - 1) / BY),
                    (unsigned)((p.nz + kz - 1) / kz));
    k_step_ws<BY, MB><<<grid, dim3(32, 2 * BY + 2), 0, st>>>(p, jstep, kz, S);
}

bool ws_supported(int by, int mb, int kz) {
    return ((by == 4 && (mb == 2 || mb == 3)) || (by == 6 && mb == 2) || (by == 8 && (mb == 1 || mb == 2))) &&
           kz >= 2 && kz <= 256;
}

cudaError_t launch_step_ws(const StepParams<float> &p, int S, int jstep, cudaStream_t st) {
    if (p.nx % 2 != 0 || !p.cEm || !p.lx.ih_h || !p.err || !p.H2 || !p.psi || !ws_supported(p.FZ_by, p.FZ_mb, p.FZ_kz))
        return cudaErrorInvalidValue;
    if (p.FZ_by == 4 && p.FZ_mb == 2) go_ws<4, 2>(p, S, jstep, st);
    else if (p.FZ_by == 4 && p.FZ_mb == 3) go_ws<4, 3>(p, S, jstep, st);
    else if (p.FZ_by == 6 && p.FZ_mb == 2) go_ws<6, 2>(p, S, jstep, st);
    else if (p.FZ_by == 8 && p.FZ_mb == 1) go_ws<8, 1>(p, S, jstep, st);
    else go_ws<8, 2>(p, S, jstep, st);
    g_launches++;
    return cudaGetLastError();
}

bool fz_supported(int by, int mb, int kz) {
    return ((by == 4 && (mb == 4 || mb == 6)) || (by == 8 && (mb == 2 || mb == 3))) && kz >= 2 && kz <= 256;
}

cudaError_t launch_step_fz(const StepParams<float> &p, int S, int jstep, cudaStream_t st) {
    if (p.nx % 2 != 0 || !p.qh || !p.qv || !p.gx.h || !p.lx.ih_h || !p.err || !p.H2 ||
        !fz_supported(p.FZ_by, p.FZ_mb, p.FZ_kz) || (p.qv != p.qh && p.qv != p.qh + p.vol))
        return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    if (p.FZ_by == 4 && p.FZ_mb == 4) e = go_fz<4, 4>(p, S, jstep, st);
    else if (p.FZ_by == 4 && p.FZ_mb == 6) e = go_fz<4, 6>(p, S, jstep, st);
    else if (p.FZ_by == 8 && p.FZ_mb == 2) e = go_fz<8, 2>(p, S, jstep, st);
    else if (p.FZ_by == 8 && p.FZ_mb == 3) e = go_fz<8, 3>(p, S, jstep, st);
    if (e != cudaSuccess) return e;
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_qcell(const GeoD &g, const float *rho, const float *rho_z, float *qh, float *qv,
                         cudaStream_t st) {
    k_qcell<<<(unsigned)((g.vol + 255) / 256), 256, 0, st>>>(g, rho, rho_z, qh, qv);
    g_launches++;
    return cudaGetLastError();
}

}  // namespace csem
