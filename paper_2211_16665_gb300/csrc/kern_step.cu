// Leap-frog time step of the fictitious-wave Maxwell system (paper Sec. 2, Eq. 4)
// on a stretched Yee grid with unsplit CPML, and the on-the-fly damped
// transform of Eq. 6 into every frequency.
//
// E lives in a ring of nslot >= M + 1 snapshots per source (E^n in slot n mod
// nslot; 2M + 1 when a block's transform overlaps the next block's steps); H and
// the CPML memory are updated in place.  Per step:
//   k_h       H^{n-1/2} -> H^{n+1/2} from E^n (slot n);
//   k_e       E^{n+1} (slot n+1) = E^n + dt/eps (curl H^{n+1/2} - J'^{n+1/2}),
//             the source term added by the thread that owns the tap's column.
// After every M steps (and once at the end for a partial block):
//   k_dft     for the M finished snapshots, sum E^n w_{k,n} over the block with
//             FMAs in registers and add the block sum to every frequency's
//             volume with Kahan compensation; sample + transform (FP64) the
//             receivers.
// The volume accumulators are read and written once per M steps instead of
// once per step, and the compensated addition runs once per block.
// Threads of k_h / k_e are laid out flat over the (j, i) plane and march KZ
// planes along z, keeping the z-neighbour in registers.
#include <algorithm>
#include <atomic>

#include "csem_internal.cuh"

namespace csem {

std::atomic<long long> g_launches{0};

template <typename R> __device__ __forceinline__ R ldg(const R *p) { return __ldg(p); }

__device__ __forceinline__ void kahan_add(double &sum, double &c, double x) {
    double y = x - c;
    double t = sum + y;
    c = (t - sum) - y;
    sum = t;
}
__device__ __forceinline__ void kahan_add(float &sum, float &c, float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

template <typename R>
__device__ __forceinline__ const R *eslot(const StepParams<R> &p, int s, int n) {
    return p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
}

template <typename R, int KZ, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_h(const StepParams<R> p, const int jstep) {
    const int t = blockIdx.x * kBlock + threadIdx.x;
    const int j = t / p.pitch;
    const int i = t - j * p.pitch;
    if (j >= p.NY || i >= p.NX) return;
    const int s = blockIdx.z;
    const int n = *p.step + jstep;
    const int k0 = blockIdx.y * KZ;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;
    const R *__restrict__ E = eslot(p, s, n);
    const R *__restrict__ Ex = E;
    const R *__restrict__ Ey = E + vol;
    const R *__restrict__ Ez = E + 2 * vol;
    R *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    R *__restrict__ Hy = Hx + vol;
    R *__restrict__ Hz = Hx + 2 * vol;
    R *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    R *__restrict__ psx = P;                         // x-slab arrays: [0]=Hy(dEz/dx) [1]=Hz(dEy/dx)
    R *__restrict__ psy = P + 6 * p.sx;              // y-slab arrays: [0]=Hx(dEz/dy) [1]=Hz(dEx/dy)
    R *__restrict__ psz = P + 6 * p.sx + 6 * p.sy;   // z-slab arrays: [0]=Hx(dEy/dz) [1]=Hy(dEx/dz)
    const int nx = p.nx, ny = p.ny, nz = p.nz, np2 = 2 * p.npml;

    const int sxh = slab_half(i, nx, p.npml);
    const int syh = slab_half(j, ny, p.npml);
    const R ihx = (i < nx) ? ldg(p.ax.ih_h + i) : R(0);
    const R ihy = (j < ny) ? ldg(p.ay.ih_h + j) : R(0);
    R bx = 0, axc = 0, by = 0, ayc = 0;
    if (sxh >= 0) { bx = ldg(p.ax.b_h + i); axc = ldg(p.ax.a_h + i); }
    if (syh >= 0) { by = ldg(p.ay.b_h + j); ayc = ldg(p.ay.a_h + j); }
    const R cH = p.cH;

    int idx = k0 * plane + j * pitch + i;
    R exc = ldg(Ex + idx), eyc = ldg(Ey + idx);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= p.NZ) break;
        const R ezc = ldg(Ez + idx);
        const bool up = (k + 1 < p.NZ);
        const R exk = up ? ldg(Ex + idx + plane) : R(0);
        const R eyk = up ? ldg(Ey + idx + plane) : R(0);
        const int szh = slab_half(k, nz, p.npml);
        const R ihz = (k < nz) ? ldg(p.az.ih_h + k) : R(0);
        R bz = 0, azc = 0;
        if (szh >= 0) { bz = ldg(p.az.b_h + k); azc = ldg(p.az.a_h + k); }

        if (j < ny && k < nz) {           // Hx at (i, j+1/2, k+1/2)
            R dEz_dy = (ldg(Ez + idx + pitch) - ezc) * ihy;
            R dEy_dz = (eyk - eyc) * ihz;
            if (syh >= 0) {
                R &ps = psy[(k * np2 + syh) * pitch + i];
                ps = by * ps + ayc * dEz_dy;
                dEz_dy += ps;
            }
            if (szh >= 0) {
                R &ps = psz[(szh * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dEy_dz;
                dEy_dz += ps;
            }
            Hx[idx] -= cH * (dEz_dy - dEy_dz);
        }
        if (i < nx && k < nz) {           // Hy at (i+1/2, j, k+1/2)
            R dEx_dz = (exk - exc) * ihz;
            R dEz_dx = (ldg(Ez + idx + 1) - ezc) * ihx;
            if (szh >= 0) {
                R &ps = psz[p.sz + (szh * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dEx_dz;
                dEx_dz += ps;
            }
            if (sxh >= 0) {
                R &ps = psx[(k * p.NY + j) * np2 + sxh];
                ps = bx * ps + axc * dEz_dx;
                dEz_dx += ps;
            }
            Hy[idx] -= cH * (dEx_dz - dEz_dx);
        }
        if (i < nx && j < ny) {           // Hz at (i+1/2, j+1/2, k)
            R dEy_dx = (ldg(Ey + idx + 1) - eyc) * ihx;
            R dEx_dy = (ldg(Ex + idx + pitch) - exc) * ihy;
            if (sxh >= 0) {
                R &ps = psx[p.sx + (k * p.NY + j) * np2 + sxh];
                ps = bx * ps + axc * dEy_dx;
                dEy_dx += ps;
            }
            if (syh >= 0) {
                R &ps = psy[p.sy + (k * np2 + syh) * pitch + i];
                ps = by * ps + ayc * dEx_dy;
                dEx_dy += ps;
            }
            Hz[idx] -= cH * (dEy_dx - dEx_dy);
        }
        exc = exk;
        eyc = eyk;
    }
}

template <typename R, int KZ, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_e(const StepParams<R> p, const int jstep) {
    const int t = blockIdx.x * kBlock + threadIdx.x;
    const int j = t / p.pitch;
    const int i = t - j * p.pitch;
    if (j >= p.NY || i >= p.NX) return;
    const int s = blockIdx.z;
    const int n = *p.step + jstep;
    const int k0 = blockIdx.y * KZ;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;
    const R *__restrict__ Eo = eslot(p, s, n);
    R *__restrict__ En = const_cast<R *>(eslot(p, s, n + 1));
    const R *__restrict__ Hx = p.H + (long long)s * 3 * vol;
    const R *__restrict__ Hy = Hx + vol;
    const R *__restrict__ Hz = Hx + 2 * vol;
    const R *__restrict__ cEx = p.cE;
    const R *__restrict__ cEy = p.cE + vol;
    const R *__restrict__ cEz = p.cE + 2 * vol;
    R *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    R *__restrict__ psx = P;                         // [2]=Ey(dHz/dx) [3]=Ez(dHy/dx)
    R *__restrict__ psy = P + 6 * p.sx;              // [2]=Ex(dHz/dy) [3]=Ez(dHx/dy)
    R *__restrict__ psz = P + 6 * p.sx + 6 * p.sy;   // [2]=Ex(dHy/dz) [3]=Ey(dHx/dz)
    const int nx = p.nx, ny = p.ny, nz = p.nz, np2 = 2 * p.npml;

    const int sxn = slab_node(i, nx, p.npml);
    const int syn = slab_node(j, ny, p.npml);
    const R ihx = ldg(p.ax.ih_n + i);
    const R ihy = ldg(p.ay.ih_n + j);
    R bx = 0, axc = 0, by = 0, ayc = 0;
    if (sxn >= 0) { bx = ldg(p.ax.b_n + i); axc = ldg(p.ax.a_n + i); }
    if (syn >= 0) { by = ldg(p.ay.b_n + j); ayc = ldg(p.ay.a_n + j); }
    const bool ix_in = (i >= 1 && i < nx), jy_in = (j >= 1 && j < ny);

    int idx = k0 * plane + j * pitch + i;
    R hxm = (k0 > 0) ? ldg(Hx + idx - plane) : R(0);
    R hym = (k0 > 0) ? ldg(Hy + idx - plane) : R(0);
#pragma unroll
    for (int kk = 0; kk < KZ; ++kk, idx += plane) {
        const int k = k0 + kk;
        if (k >= p.NZ) break;
        const R hxc = ldg(Hx + idx), hyc = ldg(Hy + idx), hzc = ldg(Hz + idx);
        const int szn = slab_node(k, nz, p.npml);
        const R ihz = ldg(p.az.ih_n + k);
        R bz = 0, azc = 0;
        if (szn >= 0) { bz = ldg(p.az.b_n + k); azc = ldg(p.az.a_n + k); }
        const bool kz_in = (k >= 1 && k < nz);

        if (i < nx && jy_in && kz_in) {   // Ex at (i+1/2, j, k)
            R dHz_dy = (hzc - ldg(Hz + idx - pitch)) * ihy;
            R dHy_dz = (hyc - hym) * ihz;
            if (syn >= 0) {
                R &ps = psy[2 * p.sy + (k * np2 + syn) * pitch + i];
                ps = by * ps + ayc * dHz_dy;
                dHz_dy += ps;
            }
            if (szn >= 0) {
                R &ps = psz[2 * p.sz + (szn * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dHy_dz;
                dHy_dz += ps;
            }
            En[idx] = ldg(Eo + idx) + ldg(cEx + idx) * (dHz_dy - dHy_dz);
        }
        if (j < ny && ix_in && kz_in) {   // Ey at (i, j+1/2, k)
            R dHx_dz = (hxc - hxm) * ihz;
            R dHz_dx = (hzc - ldg(Hz + idx - 1)) * ihx;
            if (szn >= 0) {
                R &ps = psz[3 * p.sz + (szn * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dHx_dz;
                dHx_dz += ps;
            }
            if (sxn >= 0) {
                R &ps = psx[2 * p.sx + (k * p.NY + j) * np2 + sxn];
                ps = bx * ps + axc * dHz_dx;
                dHz_dx += ps;
            }
            En[vol + idx] = ldg(Eo + vol + idx) + ldg(cEy + idx) * (dHx_dz - dHz_dx);
        }
        if (k < nz && ix_in && jy_in) {   // Ez at (i, j, k+1/2)
            R dHy_dx = (hyc - ldg(Hy + idx - 1)) * ihx;
            R dHx_dy = (hxc - ldg(Hx + idx - pitch)) * ihy;
            if (sxn >= 0) {
                R &ps = psx[3 * p.sx + (k * p.NY + j) * np2 + sxn];
                ps = bx * ps + axc * dHy_dx;
                dHy_dx += ps;
            }
            if (syn >= 0) {
                R &ps = psy[3 * p.sy + (k * np2 + syn) * pitch + i];
                ps = by * ps + ayc * dHx_dy;
                dHx_dy += ps;
            }
            En[2 * vol + idx] = ldg(Eo + 2 * vol + idx) + ldg(cEz + idx) * (dHy_dx - dHx_dy);
        }
        hxm = hxc;
        hym = hyc;
    }
    // source term E^{n+1} -= dt/eps J'^{n+1/2}: this thread owns its column's taps
    if (p.colmap) {
        const int2 cm = p.colmap[s * p.colmap_stride + j * pitch + i];
        for (int u = cm.x; u < cm.x + cm.y; ++u) {
            const Tap tp = p.itaps[(long long)s * p.itap_stride + u];
            const int k = (int)(tp.idx / plane);
            if (k < k0 || k >= k0 + KZ) continue;
            const double *cf = p.coef + ((long long)s * p.n_emit + tp.emit) * p.J;
            const double *T = p.T + (long long)n * p.J;
            double amp = 0.0;
            for (int jj = 0; jj < p.J; ++jj) amp += cf[jj] * T[jj];
            const int o = tp.comp * vol + (int)tp.idx;
            const double add = -(double)p.cE[o] * tp.w * amp;   // dt/eps at the tap's edge
            if (add != 0.0) En[o] += (R)add;
        }
    }
}

// Transform of the snapshots n0 .. n0+cnt-1 (n0 = *step + n0_off).
// Blocks [0, S): receivers, one block per source (they start first);
// blocks [S, S + nvb*3*S): volume entries (block -> (vb, c, s)).  CNT > 0:
// cnt is a multiple of CNT and the snapshots are read in unrolled groups of
// CNT; CNT = 0: any cnt, one snapshot at a time.
template <typename R, bool VOL, bool KAHAN, int CNT>
__global__ void __launch_bounds__(kBlock) k_dft(const StepParams<R> p, const PointParams<R> q, const int n0_off,
                                                const int cnt_rt, const int nvb, const int S) {
    typedef typename C2<R>::T R2;
    __shared__ R2 wsh[kMaxBlockSteps * kMaxFreq];
    const int n0 = *p.step + n0_off;
    if (n0 < 0) return;               // a deferred flush before the first block: nothing to transform
    const int cnt = cnt_rt;
    const int nrec_blocks = q.n_rec > 0 ? S : 0;
    const int blk = blockIdx.x;
    if (blk < nrec_blocks) {
        const int s = blk;
        const R *ring = p.ering + (long long)s * p.ering_stride;
        for (int r = threadIdx.x; r < q.n_rec; r += blockDim.x) {
            const Tap *tp = q.rtaps + (long long)r * 8;
            double2 a[kMaxFreq];
            double2 *dst = q.racc + ((long long)s * q.n_rec + r) * q.nf;
            for (int f = 0; f < q.nf; ++f) a[f] = dst[f];
            for (int m = 0; m < cnt; ++m) {
                const int n = n0 + m;
                const R *E = ring + (long long)(n % p.nslot) * 3 * p.vol;
                double v = 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u) v += tp[u].w * (double)E[(long long)tp[u].comp * p.vol + tp[u].idx];
                const double2 *w = q.w64 + (long long)n * q.nf;
                for (int f = 0; f < q.nf; ++f) {
                    a[f].x += v * w[f].x;
                    a[f].y += v * w[f].y;
                }
                if (q.trace) q.trace[((long long)s * q.n_rec + r) * q.nt + n] = v;
            }
            for (int f = 0; f < q.nf; ++f) dst[f] = a[f];
        }
        return;
    }
    if constexpr (VOL) {
    for (int u = threadIdx.x; u < cnt * p.nf; u += blockDim.x) wsh[u] = p.w[(long long)n0 * p.nf + u];
    __syncthreads();
    const int vblk = blk - nrec_blocks;
    const int vb = vblk % nvb;
    const int c = (vblk / nvb) % 3;
    const int s = vblk / (nvb * 3);
    const long long idx = (long long)vb * kBlock + threadIdx.x;
    if (idx >= p.vol) return;
    R2 *__restrict__ A = p.acc + ((long long)s * 3 + c) * p.nf * p.vol + idx;
    R2 *__restrict__ C = KAHAN ? p.comp + ((long long)s * 3 + c) * p.nf * p.vol + idx : nullptr;
    const R *__restrict__ base = p.ering + (long long)s * p.ering_stride + (long long)c * p.vol + idx;
    const long long slot = 3 * p.vol;
    R2 acc[kMaxFreq], cmp[kMaxFreq];
#pragma unroll
    for (int f = 0; f < kMaxFreq; ++f)
        if (f < p.nf) {
            acc[f] = A[(long long)f * p.vol];
            if (KAHAN) cmp[f] = C[(long long)f * p.vol];
        }
    // block sum of the products with plain FMAs, then one compensated addition
    // of the block sum to the running accumulator
    R2 bs[kMaxFreq];
#pragma unroll
    for (int f = 0; f < kMaxFreq; ++f) bs[f].x = bs[f].y = R(0);
    if (CNT > 0) {
        // whole groups of CNT snapshots: every load of a group is issued before its FMAs
        int sl = n0 % p.nslot;
        for (int g = 0; g < cnt; g += CNT) {
            R e[CNT > 0 ? CNT : 1];
#pragma unroll
            for (int m = 0; m < CNT; ++m) {
                e[m] = ldg(base + (long long)sl * slot);
                sl = (sl + 1 == p.nslot) ? 0 : sl + 1;
            }
#pragma unroll
            for (int m = 0; m < CNT; ++m)
#pragma unroll
                for (int f = 0; f < kMaxFreq; ++f)
                    if (f < p.nf) {
                        const R2 w = wsh[(g + m) * p.nf + f];
                        bs[f].x = fma(e[m], w.x, bs[f].x);
                        bs[f].y = fma(e[m], w.y, bs[f].y);
                    }
        }
    } else {
        for (int m = 0; m < cnt; ++m) {
            const R e = ldg(base + (long long)((n0 + m) % p.nslot) * slot);
#pragma unroll
            for (int f = 0; f < kMaxFreq; ++f)
                if (f < p.nf) {
                    const R2 w = wsh[m * p.nf + f];
                    bs[f].x = fma(e, w.x, bs[f].x);
                    bs[f].y = fma(e, w.y, bs[f].y);
                }
        }
    }
#pragma unroll
    for (int f = 0; f < kMaxFreq; ++f)
        if (f < p.nf) {
            if (KAHAN) {
                kahan_add(acc[f].x, cmp[f].x, bs[f].x);
                kahan_add(acc[f].y, cmp[f].y, bs[f].y);
            } else {
                acc[f].x += bs[f].x;
                acc[f].y += bs[f].y;
            }
        }
#pragma unroll
    for (int f = 0; f < kMaxFreq; ++f)
        if (f < p.nf) {
            A[(long long)f * p.vol] = acc[f];
            if (KAHAN) C[(long long)f * p.vol] = cmp[f];
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk-copy flush (FP32): the tensor-memory-access engine streams each block's
// rows -- MS snapshots of 256 lattice entries and the accumulator (and Kahan)
// rows -- into shared memory with cp.async.bulk on one mbarrier, so every byte
// of the block is in flight at once with few registers.  The wait on the
// barrier is bounded (about a second): on timeout the block raises the flush
// bit of *err, waits once more (bounded) for its own copies and returns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    uint64_t g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(g), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}


// Packed FP32 pairs for the flush sums: a complex accumulator (re, im) or a weight pair in
// one 64-bit register, and a real value duplicated into both lanes.  fma.rn.f32x2 does one
// fused multiply-add per lane, each rounded to nearest once, so a sum built with it equals
// the sum of the same fmaf calls bit for bit, with half the instructions.
__device__ __forceinline__ uint64_t dup_f32x2(float v) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ void fma_f32x2(uint64_t &acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ float2 unpack_f32x2(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// Receiver transforms of source s over the ms snapshots from step n0 (FP64 sums of the
// eight interpolation taps of each receiver), one receiver per thread.
__device__ __forceinline__ void dft_receivers(const StepParams<float> &p, const PointParams<float> &q, int n0, int ms,
                                              int s) {
    const float *ring = p.ering + (long long)s * p.ering_stride;
    for (int r = threadIdx.x; r < q.n_rec; r += blockDim.x) {
        const Tap *tp = q.rtaps + (long long)r * 8;
        double2 a[kMaxFreq];
        double2 *dst = q.racc + ((long long)s * q.n_rec + r) * q.nf;
        for (int f = 0; f < q.nf; ++f) a[f] = dst[f];
        for (int m = 0; m < ms; ++m) {
            const int n = n0 + m;
            const float *E = ring + (long long)(n % p.nslot) * 3 * p.vol;
            double v = 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u) v += tp[u].w * (double)E[(long long)tp[u].comp * p.vol + tp[u].idx];
            const double2 *w = q.w64 + (long long)n * q.nf;
            for (int f = 0; f < q.nf; ++f) {
                a[f].x += v * w[f].x;
                a[f].y += v * w[f].y;
            }
            if (q.trace) q.trace[((long long)s * q.n_rec + r) * q.nt + n] = v;
        }
        for (int f = 0; f < q.nf; ++f) dst[f] = a[f];
    }
}

// resident blocks per SM that the shared memory allows (MS snapshots of 1 KB + accumulators)
template <int MS> constexpr int bulk_minb() { return MS <= 16 ? 6 : 4; }   // 16 or 32 snapshots
constexpr int kBulkThreads = 128;       // two lattice entries per thread, 256 per block
__host__ __device__ constexpr int nf_pad(int nf) { return nf <= 2 ? 2 : (nf <= 4 ? 4 : 8); }

// Each thread sums its two entries' MS snapshots into NF frequencies (NF a
// compile-time bound, the weights of frequencies >= nf are zero and their sums
// are dropped), reading each snapshot pair with one 8-byte load and each pair
// of complex weights with one 16-byte broadcast, and summing with packed FMAs.  One warp waits on the
// barrier; the others wait at __syncthreads without issuing.
template <bool KAHAN, int MS, int NF>
__global__ void __launch_bounds__(kBulkThreads, bulk_minb<MS>()) k_dft_bulk(const StepParams<float> p,
                                                                            const PointParams<float> q,
                                                                            const int n0_off, const int nvb,
                                                                            const int S, int *err) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int bad;
    extern __shared__ __align__(128) unsigned char smem[];
    float *ring_s = reinterpret_cast<float *>(smem);                        // [MS][256]
    float2 *acc_s = reinterpret_cast<float2 *>(ring_s + MS * kBlock);       // [nf][256]
    float2 *cmp_s = acc_s + p.nf * kBlock;                                  // [nf][256] (Kahan)
    float2 *w_s = cmp_s + (KAHAN ? p.nf * kBlock : 0);                      // [MS][NF], zero past nf
    const int n0 = *p.step + n0_off;
    if (n0 < 0) return;               // a deferred flush before the first block: nothing to transform
    const int nrec_blocks = q.n_rec > 0 ? S : 0;
    const int blk = blockIdx.x;
    if (blk < nrec_blocks) {          // receivers: same as the register flush
        dft_receivers(p, q, n0, MS, blk);
        return;
    }
    const int vblk = blk - nrec_blocks;
    const int vb = vblk % nvb;
    const int c = (vblk / nvb) % 3;
    const int s = vblk / (nvb * 3);
    const long long i0 = (long long)vb * kBlock;
    const int rows = (int)min((long long)kBlock, p.vol - i0);      // a multiple of 8 entries
    float2 *A = p.acc + ((long long)s * 3 + c) * p.nf * p.vol + i0;
    float2 *C = KAHAN ? p.comp + ((long long)s * 3 + c) * p.nf * p.vol + i0 : nullptr;
    const float *ring = p.ering + (long long)s * p.ering_stride + (long long)c * p.vol + i0;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        bad = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t rb = (uint32_t)rows * sizeof(float), cb = (uint32_t)rows * sizeof(float2);
        mbar_expect_tx(&bar, MS * rb + p.nf * cb * (KAHAN ? 2u : 1u) + (uint32_t)p.fault_tx);
        int sl = n0 % p.nslot;
        for (int m = 0; m < MS; ++m) {
            bulk_g2s(ring_s + m * kBlock, ring + (long long)sl * 3 * p.vol, rb, &bar);
            sl = (sl + 1 == p.nslot) ? 0 : sl + 1;
        }
        for (int f = 0; f < p.nf; ++f) {
            bulk_g2s(acc_s + f * kBlock, A + (long long)f * p.vol, cb, &bar);
            if (KAHAN) bulk_g2s(cmp_s + f * kBlock, C + (long long)f * p.vol, cb, &bar);
        }
    }
    for (int u = threadIdx.x; u < MS * NF; u += blockDim.x) {
        const int m = u / NF, f = u - m * NF;
        w_s[u] = (f < p.nf) ? p.w[(long long)(n0 + m) * p.nf + f] : make_float2(0.f, 0.f);
    }
    if (threadIdx.x < 32) {
        if (!mbar_wait_bounded(&bar, 0)) {
            if (threadIdx.x == 0) {
                atomicOr(err, kErrFlushWait);
                bad = 1;
            }
            mbar_wait_bounded(&bar, 0);     // once more, so no copy can still be landing at exit
        }
    }
    __syncthreads();
    if (bad) return;
    const int t2 = 2 * threadIdx.x;
    if (t2 >= rows) return;
    uint64_t p0[NF], p1[NF];            // packed (re, im) block sums of entries t2, t2 + 1
#pragma unroll
    for (int f = 0; f < NF; ++f) p0[f] = p1[f] = 0ull;
    const ulonglong2 *w2 = reinterpret_cast<const ulonglong2 *>(w_s);
#pragma unroll 4
    for (int m = 0; m < MS; ++m) {
        const float2 e = *reinterpret_cast<const float2 *>(ring_s + m * kBlock + t2);
        const uint64_t ex = dup_f32x2(e.x), ey = dup_f32x2(e.y);
#pragma unroll
        for (int g = 0; g < NF / 2; ++g) {
            const ulonglong2 w = w2[m * (NF / 2) + g];   // (re, im) of frequencies 2g and 2g+1
            fma_f32x2(p0[2 * g], ex, w.x);
            fma_f32x2(p0[2 * g + 1], ex, w.y);
            fma_f32x2(p1[2 * g], ey, w.x);
            fma_f32x2(p1[2 * g + 1], ey, w.y);
        }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f >= p.nf) break;
        const float2 s0 = unpack_f32x2(p0[f]), s1 = unpack_f32x2(p1[f]);
        float4 a = *reinterpret_cast<const float4 *>(acc_s + f * kBlock + t2);   // entries t2, t2+1
        if (KAHAN) {
            float4 cc = *reinterpret_cast<const float4 *>(cmp_s + f * kBlock + t2);
            kahan_add(a.x, cc.x, s0.x);
            kahan_add(a.y, cc.y, s0.y);
            kahan_add(a.z, cc.z, s1.x);
            kahan_add(a.w, cc.w, s1.y);
            *reinterpret_cast<float4 *>(C + (long long)f * p.vol + t2) = cc;
        } else {
            a.x += s0.x;
            a.y += s0.y;
            a.z += s1.x;
            a.w += s1.y;
        }
        *reinterpret_cast<float4 *>(A + (long long)f * p.vol + t2) = a;
    }
}

// Streamed flush of kStMS = 64 or 128 snapshots.  Holding all 64 snapshot rows of
// a block in shared memory (64 KB) leaves two blocks per SM, and a block computes
// only after its last copy landed.  Here the snapshots stream through kStN stages of
// kStG rows each (one mbarrier per stage, 32 KB in all): while the block sums
// the rows of one stage, the copies of the next kStN - 1 stages are in flight,
// and four blocks fit an SM.  The accumulators (and compensation) arrive on a
// barrier of their own (with eight frequencies they are read from global memory
// at the end instead, see stream_stages_acc) and are added to once, at the end, as in k_dft_bulk;
// the sums are the ones k_dft_bulk would form over the same snapshots, in the same order.
// Each thread waits on each stage's barrier itself (bounded); a give-up
// anywhere ends the loop for the whole block (__syncthreads_or), thread 0 then
// waits (bounded) for every copy it issued that nobody consumed, and the block
// returns with the flush bit of *err raised.
constexpr int kStG = 8;                 // snapshot rows per stage
constexpr int kStN = 4;                 // stages (a power of two)
// With up to four frequencies the accumulator rows are staged in shared memory (on their own
// barrier, while the snapshots stream); with eight they would take 32 KB and leave three blocks
// per SM, so each thread reads its accumulators from global memory at the end instead and five
// blocks fit.
__host__ __device__ constexpr bool stream_stages_acc(int nf_padded) { return nf_padded <= 4; }
__host__ __device__ constexpr int stream_minb(int nf_padded) { return stream_stages_acc(nf_padded) ? 3 : 5; }

template <bool KAHAN, int NF, int kStMS>
__global__ void __launch_bounds__(kBulkThreads, stream_minb(NF)) k_dft_stream(const StepParams<float> p,
                                                                              const PointParams<float> q,
                                                                              const int n0_off, const int nvb,
                                                                              const int S, int *err) {
    constexpr int NCH = kStMS / kStG;
    constexpr bool SACC = stream_stages_acc(NF);
    __shared__ __align__(8) uint64_t full[kStN];
    __shared__ __align__(8) uint64_t abar;
    extern __shared__ __align__(128) unsigned char smem[];
    float *st_s = reinterpret_cast<float *>(smem);                          // [kStN][kStG][256]
    float2 *acc_s = reinterpret_cast<float2 *>(st_s + kStN * kStG * kBlock);  // [nf][256] (SACC)
    float2 *cmp_s = acc_s + (SACC ? p.nf * kBlock : 0);                     // [nf][256] (SACC, Kahan)
    float2 *w_s = cmp_s + (SACC && KAHAN ? p.nf * kBlock : 0);              // [kStMS][NF], zero past nf
    const int n0 = *p.step + n0_off;
    if (n0 < 0) return;
    const int nrec_blocks = q.n_rec > 0 ? S : 0;
    const int blk = blockIdx.x;
    if (blk < nrec_blocks) {
        dft_receivers(p, q, n0, kStMS, blk);
        return;
    }
    const int vblk = blk - nrec_blocks;
    const int vb = vblk % nvb;
    const int c = (vblk / nvb) % 3;
    const int s = vblk / (nvb * 3);
    const long long i0 = (long long)vb * kBlock;
    const int rows = (int)min((long long)kBlock, p.vol - i0);      // a multiple of 8 entries
    float2 *A = p.acc + ((long long)s * 3 + c) * p.nf * p.vol + i0;
    float2 *C = KAHAN ? p.comp + ((long long)s * 3 + c) * p.nf * p.vol + i0 : nullptr;
    const float *ring = p.ering + (long long)s * p.ering_stride + (long long)c * p.vol + i0;
    const uint32_t rb = (uint32_t)rows * sizeof(float), cb = (uint32_t)rows * sizeof(float2);
    if (threadIdx.x == 0) {
        for (int u = 0; u < kStN; ++u) mbar_init(&full[u], 1);
        mbar_init(&abar, 1);
    }
    __syncthreads();
    int issued = 0;                     // chunks issued (meaningful in thread 0)
    auto issue = [&](int ch) {          // snapshots ch*kStG .. into stage ch % kStN
        const int u = ch & (kStN - 1);
        mbar_expect_tx(&full[u], kStG * rb + (ch == 0 ? (uint32_t)p.fault_tx : 0u));
        int sl = (n0 + ch * kStG) % p.nslot;
        for (int g = 0; g < kStG; ++g) {
            bulk_g2s(st_s + (u * kStG + g) * kBlock, ring + (long long)sl * 3 * p.vol, rb, &full[u]);
            sl = (sl + 1 == p.nslot) ? 0 : sl + 1;
        }
        issued = ch + 1;
    };
    if (threadIdx.x == 0) {
        for (int ch = 0; ch < kStN; ++ch) issue(ch);
        if (SACC) {
            mbar_expect_tx(&abar, p.nf * cb * (KAHAN ? 2u : 1u));
            for (int f = 0; f < p.nf; ++f) {
                bulk_g2s(acc_s + f * kBlock, A + (long long)f * p.vol, cb, &abar);
                if (KAHAN) bulk_g2s(cmp_s + f * kBlock, C + (long long)f * p.vol, cb, &abar);
            }
        }
    }
    for (int u = threadIdx.x; u < kStMS * NF; u += blockDim.x) {
        const int m = u / NF, f = u - m * NF;
        w_s[u] = (f < p.nf) ? p.w[(long long)(n0 + m) * p.nf + f] : make_float2(0.f, 0.f);
    }
    const int t2 = 2 * threadIdx.x;
    const bool mine = t2 < rows;
    uint64_t p0[NF], p1[NF];            // packed (re, im) block sums of entries t2, t2 + 1
#pragma unroll
    for (int f = 0; f < NF; ++f) p0[f] = p1[f] = 0ull;
    const ulonglong2 *w2 = reinterpret_cast<const ulonglong2 *>(w_s);
    bool ok = true;
    int ch = 0;
    for (; ch < NCH; ++ch) {
        const int u = ch & (kStN - 1);
        if (ok) ok = mbar_wait_bounded(&full[u], (uint32_t)(ch / kStN) & 1u);
        // every thread has finished chunk ch - 1: its stage takes chunk ch - 1 + kStN
        if (__syncthreads_or(!ok)) break;
        if (threadIdx.x == 0 && ch >= 1 && ch - 1 + kStN < NCH) issue(ch - 1 + kStN);
        if (!mine) continue;
        const float *sg = st_s + u * kStG * kBlock + t2;
#pragma unroll
        for (int g = 0; g < kStG; ++g) {
            const float2 e = *reinterpret_cast<const float2 *>(sg + g * kBlock);
            const uint64_t ex = dup_f32x2(e.x), ey = dup_f32x2(e.y);
            const int m = ch * kStG + g;
#pragma unroll
            for (int h = 0; h < NF / 2; ++h) {
                const ulonglong2 w = w2[m * (NF / 2) + h];   // (re, im) of frequencies 2h and 2h+1
                fma_f32x2(p0[2 * h], ex, w.x);
                fma_f32x2(p0[2 * h + 1], ex, w.y);
                fma_f32x2(p1[2 * h], ey, w.x);
                fma_f32x2(p1[2 * h + 1], ey, w.y);
            }
        }
    }
    const bool done = (ch == NCH);
    if (SACC && done && ok) ok = mbar_wait_bounded(&abar, 0);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(err, kErrFlushWait);
            // copies issued and not consumed: chunks ch .. issued - 1 (each in its own stage), and
            // the accumulators; a wait that already completed returns at once
            for (int x = ch; x < issued; ++x) mbar_wait_bounded(&full[x & (kStN - 1)], (uint32_t)(x / kStN) & 1u);
            if (SACC) mbar_wait_bounded(&abar, 0);
        }
        return;
    }
    if (!mine) return;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        if (f >= p.nf) break;
        const float2 s0 = unpack_f32x2(p0[f]), s1 = unpack_f32x2(p1[f]);
        // entries t2, t2+1
        float4 a = SACC ? *reinterpret_cast<const float4 *>(acc_s + f * kBlock + t2)
                        : *reinterpret_cast<const float4 *>(A + (long long)f * p.vol + t2);
        if (KAHAN) {
            float4 cc = SACC ? *reinterpret_cast<const float4 *>(cmp_s + f * kBlock + t2)
                             : *reinterpret_cast<const float4 *>(C + (long long)f * p.vol + t2);
            kahan_add(a.x, cc.x, s0.x);
            kahan_add(a.y, cc.y, s0.y);
            kahan_add(a.z, cc.z, s1.x);
            kahan_add(a.w, cc.w, s1.y);
            *reinterpret_cast<float4 *>(C + (long long)f * p.vol + t2) = cc;
        } else {
            a.x += s0.x;
            a.y += s0.y;
            a.z += s1.x;
            a.w += s1.y;
        }
        *reinterpret_cast<float4 *>(A + (long long)f * p.vol + t2) = a;
    }
}

size_t stream_smem_bytes(int nf, bool kahan, int ms) {
    const size_t acc = stream_stages_acc(nf_pad(nf)) ? (size_t)nf * kBlock * sizeof(float2) * (kahan ? 2 : 1) : 0;
    return (size_t)kStN * kStG * kBlock * sizeof(float) + acc + (size_t)ms * nf_pad(nf) * sizeof(float2);
}

size_t bulk_smem_bytes(int ms, int nf, bool kahan) {
    return (size_t)ms * kBlock * sizeof(float) + (size_t)nf * kBlock * sizeof(float2) * (kahan ? 2 : 1) +
           (size_t)ms * nf_pad(nf) * sizeof(float2);
}

namespace {
template <bool KAHAN, int MS, int NF>
cudaError_t bulk_attr(int bytes) {
    return cudaFuncSetAttribute(k_dft_bulk<KAHAN, MS, NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <int MS>
cudaError_t bulk_attr_ms(int bytes) {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {bulk_attr<true, MS, 2>(bytes), bulk_attr<true, MS, 4>(bytes), bulk_attr<true, MS, 8>(bytes),
                          bulk_attr<false, MS, 2>(bytes), bulk_attr<false, MS, 4>(bytes), bulk_attr<false, MS, 8>(bytes)})
        if (r != cudaSuccess) e = r;
    return e;
}
template <bool KAHAN, int NF, int MS>
cudaError_t stream_attr(int bytes) {
    return cudaFuncSetAttribute(k_dft_stream<KAHAN, NF, MS>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}
template <int MS>
cudaError_t stream_attr_ms(int bytes) {
    cudaError_t e = cudaSuccess;
    for (cudaError_t r : {stream_attr<true, 2, MS>(bytes), stream_attr<true, 4, MS>(bytes), stream_attr<true, 8, MS>(bytes),
                          stream_attr<false, 2, MS>(bytes), stream_attr<false, 4, MS>(bytes), stream_attr<false, 8, MS>(bytes)})
        if (r != cudaSuccess) e = r;
    return e;
}
template <bool KAHAN, int MS>
void stream_go(const StepParams<float> &p, const PointParams<float> &q, int S, int n0_off, int nvb, int nblk, size_t sm,
               int *err, cudaStream_t st) {
    const int np = nf_pad(p.nf);
    if (np == 2) k_dft_stream<KAHAN, 2, MS><<<nblk, kBulkThreads, sm, st>>>(p, q, n0_off, nvb, S, err);
    else if (np == 4) k_dft_stream<KAHAN, 4, MS><<<nblk, kBulkThreads, sm, st>>>(p, q, n0_off, nvb, S, err);
    else k_dft_stream<KAHAN, 8, MS><<<nblk, kBulkThreads, sm, st>>>(p, q, n0_off, nvb, S, err);
}
template <bool KAHAN, int MS>
void bulk_go(const StepParams<float> &p, const PointParams<float> &q, int S, int n0_off, int nvb, int nblk, size_t sm,
             int *err, cudaStream_t st) {
    const int np = nf_pad(p.nf);
    if (np == 2) k_dft_bulk<KAHAN, MS, 2><<<nblk, kBulkThreads, sm, st>>>(p, q, n0_off, nvb, S, err);
    else if (np == 4) k_dft_bulk<KAHAN, MS, 4><<<nblk, kBulkThreads, sm, st>>>(p, q, n0_off, nvb, S, err);
    else k_dft_bulk<KAHAN, MS, 8><<<nblk, kBulkThreads, sm, st>>>(p, q, n0_off, nvb, S, err);
}
}  // namespace

cudaError_t prepare_bulk_flush() {
    const int big = (int)bulk_smem_bytes(32, kMaxFreq, true);
    cudaError_t e = bulk_attr_ms<32>(big);
    if (e == cudaSuccess) e = bulk_attr_ms<16>(big);
    const int sbig = (int)std::max(stream_smem_bytes(4, true, 128), stream_smem_bytes(kMaxFreq, true, 128));
    if (e == cudaSuccess) e = stream_attr_ms<64>(sbig);
    if (e == cudaSuccess) e = stream_attr_ms<128>(sbig);
    return e;
}

cudaError_t launch_dft_bulk(const StepParams<float> &p, const PointParams<float> &q, int S, int n0_off, int cnt,
                            bool kahan, int *err, cudaStream_t st) {
    const int nvb = (int)((p.vol + kBlock - 1) / kBlock);
    const int nblk = nvb * 3 * S + (q.n_rec > 0 ? S : 0);
    const size_t sm = bulk_smem_bytes(cnt, p.nf, kahan);
    if (cnt == 64 || cnt == 128) {    // 64 or 128 snapshots stream through a 4-stage ring (k_dft_stream)
        const size_t ssm = stream_smem_bytes(p.nf, kahan, cnt);
        if (cnt == 64) {
            if (kahan) stream_go<true, 64>(p, q, S, n0_off, nvb, nblk, ssm, err, st);
            else stream_go<false, 64>(p, q, S, n0_off, nvb, nblk, ssm, err, st);
        } else {
            if (kahan) stream_go<true, 128>(p, q, S, n0_off, nvb, nblk, ssm, err, st);
            else stream_go<false, 128>(p, q, S, n0_off, nvb, nblk, ssm, err, st);
        }
    } else if (cnt == 32) {
        if (kahan) bulk_go<true, 32>(p, q, S, n0_off, nvb, nblk, sm, err, st);
        else bulk_go<false, 32>(p, q, S, n0_off, nvb, nblk, sm, err, st);
    } else if (cnt == 16) {
        if (kahan) bulk_go<true, 16>(p, q, S, n0_off, nvb, nblk, sm, err, st);
        else bulk_go<false, 16>(p, q, S, n0_off, nvb, nblk, sm, err, st);
    } else {
        return cudaErrorInvalidValue;
    }
    g_launches++;
    return cudaGetLastError();
}

__global__ void k_advance(int *step, int by) { *step += by; }

template <typename R, int KZ, int MB>
void launch_hz(const StepParams<R> &p, dim3 grid, int jstep, cudaStream_t st, bool h) {
    if (h) k_h<R, KZ, MB><<<grid, kBlock, 0, st>>>(p, jstep);
    else k_e<R, KZ, MB><<<grid, kBlock, 0, st>>>(p, jstep);
}

template <typename R, int MB>
bool launch_kz(const StepParams<R> &p, dim3 grid, int jstep, cudaStream_t st, bool h, int kz) {
    switch (kz) {
        case 1: launch_hz<R, 1, MB>(p, grid, jstep, st, h); return true;
        case 2: launch_hz<R, 2, MB>(p, grid, jstep, st, h); return true;
        case 4: launch_hz<R, 4, MB>(p, grid, jstep, st, h); return true;
        case 8: launch_hz<R, 8, MB>(p, grid, jstep, st, h); return true;
        default: return false;
    }
}

template <typename R>
cudaError_t launch_field(const StepParams<R> &p, int S, int jstep, cudaStream_t st, bool h, int kz, int mb) {
    if constexpr (sizeof(R) == 4) {
        const int ty = h ? p.TMA_h : p.TMA_e;
        if (h ? p.LEAN_h : p.LEAN_e) return launch_field_lean(p, S, jstep, st, h, h ? p.LEAN_h : p.LEAN_e, kz, mb);
        if (ty > 0) return launch_field_tma(p, S, jstep, st, h, kz, ty, p.err);
        if (h ? p.VEC_h : p.VEC_e) return launch_field_vec(p, S, jstep, st, h, kz, mb);
    }
    const long long plane_threads = (long long)p.NY * p.pitch;
    dim3 grid((unsigned)((plane_threads + kBlock - 1) / kBlock), (unsigned)((p.NZ + kz - 1) / kz), (unsigned)S);
    bool ok = false;
    if (mb == 4) ok = launch_kz<R, 4>(p, grid, jstep, st, h, kz);
    else if (mb == 6) ok = launch_kz<R, 6>(p, grid, jstep, st, h, kz);
    else if (mb == 8) ok = launch_kz<R, 8>(p, grid, jstep, st, h, kz);
    if (!ok) return cudaErrorInvalidValue;
    g_launches++;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_step(const StepParams<R> &p, const PointParams<R> &q, int S, int jstep, cudaStream_t st,
                        int which) {
    (void)q;
    cudaError_t e = cudaSuccess;
    if constexpr (sizeof(R) == 4) {
        if (p.FZ_by > 0 && (which & 5) == 5)
            return p.FZ_ws ? launch_step_ws(p, S, jstep, st) : launch_step_fz(p, S, jstep, st);
        if (p.WAVE_lag > 0 && (which & 5) == 5) return launch_step_wave(p, S, jstep, st);
    }
    if (p.fused_kz > 0 && (which & 5) == 5) return launch_fused<R>(p, S, jstep, p.fused_kz, st);
    if (which & 1) e = launch_field<R>(p, S, jstep, st, true, p.KZ_h, p.MB_h);
    if (e == cudaSuccess && (which & 4)) e = launch_field<R>(p, S, jstep, st, false, p.KZ_e, p.MB_e);
    return e;
}

template <typename R>
cudaError_t launch_dft(const StepParams<R> &p, const PointParams<R> &q, int S, int n0_off, int cnt, bool vol,
                       bool kahan, cudaStream_t st) {
    const int nvb = (int)((p.vol + kBlock - 1) / kBlock);
    const int nblk = (vol ? nvb * 3 * S : 0) + (q.n_rec > 0 ? S : 0);
    if (nblk == 0 || cnt <= 0) return cudaSuccess;
    // the weights of all cnt snapshots and nf frequencies are staged in shared memory at once
    if (cnt > kMaxBlockSteps || q.nf > kMaxFreq || p.nf > kMaxFreq) return cudaErrorInvalidValue;
    const bool full = (cnt % 16 == 0);
    if (!vol) k_dft<R, false, false, 0><<<nblk, kBlock, 0, st>>>(p, q, n0_off, cnt, nvb, S);
    else if (kahan && full) k_dft<R, true, true, 16><<<nblk, kBlock, 0, st>>>(p, q, n0_off, cnt, nvb, S);
    else if (kahan) k_dft<R, true, true, 0><<<nblk, kBlock, 0, st>>>(p, q, n0_off, cnt, nvb, S);
    else if (full) k_dft<R, true, false, 16><<<nblk, kBlock, 0, st>>>(p, q, n0_off, cnt, nvb, S);
    else k_dft<R, true, false, 0><<<nblk, kBlock, 0, st>>>(p, q, n0_off, cnt, nvb, S);
    g_launches++;
    return cudaGetLastError();
}

cudaError_t launch_advance(int *step, int by, cudaStream_t st) {
    k_advance<<<1, 1, 0, st>>>(step, by);
    g_launches++;
    return cudaGetLastError();
}

template cudaError_t launch_step<float>(const StepParams<float> &, const PointParams<float> &, int, int, cudaStream_t,
                                        int);
template cudaError_t launch_step<double>(const StepParams<double> &, const PointParams<double> &, int, int,
                                         cudaStream_t, int);
template cudaError_t launch_dft<float>(const StepParams<float> &, const PointParams<float> &, int, int, int, bool,
                                       bool, cudaStream_t);
template cudaError_t launch_dft<double>(const StepParams<double> &, const PointParams<double> &, int, int, int, bool,
                                        bool, cudaStream_t);

}  // namespace csem
