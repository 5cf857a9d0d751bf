// One fused leap-frog step (paper Sec. 2, Eq. 4): H^{n-1/2} -> H^{n+1/2} and
// E^n -> E^{n+1} in a single kernel, with source injection.
//
// A block owns a TX x TY tile of cells (32 x 16, 256 threads, two rows per
// thread) and marches KZ planes along z.  Per plane k:
//   * E^n planes k and k+1 (tile + one cell of halo on every side) and H^{n-1/2}
//     plane k (tile + low halo) are already in shared memory -- they were
//     prefetched with cp.async one iteration earlier, overlapping the compute;
//   * H^{n+1/2} is computed on the tile and on its low x / y halo (the halo
//     values are recomputed here rather than read, since the neighbour block
//     may already have replaced them) and kept in shared memory for plane k and
//     k-1; the tile's values go to the output H buffer;
//   * E^{n+1} on the tile reads its curl H neighbours from shared memory.
// H and the CPML memory of the H update are double-buffered (read the buffer
// of parity n, write the other), so no block ever reads a value another block
// has already advanced.  The work domain is the cell range [0,nx) x [0,ny) x
// [0,nz): every updated E edge and every H face that can change lies in it.
#include "csem_internal.cuh"

namespace csem {

namespace {

constexpr int TX = 32, TY = 16, BY = 8;        // tile, threads per block = TX * BY
constexpr int EX = TX + 2, EY = TY + 2;        // E tile with halo: i0-1 .. i0+TX, j0-1 .. j0+TY
constexpr int HX = TX + 1, HY = TY + 1;        // H tile with low halo: i0-1 .. i0+TX-1, j0-1 .. j0+TY-1
constexpr int EPL = EX * EY, HPL = HX * HY;    // entries per plane and component

template <typename R>
__device__ __forceinline__ void cp_async_or_zero(R *dst, const R *src, bool valid) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const int n = valid ? (int)sizeof(R) : 0;   // 0 bytes read: the destination is zero-filled
    if (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

}  // namespace

size_t fused_smem_bytes(int real_size) { return (size_t)real_size * (3 * 3 * EPL + 2 * 3 * HPL + 2 * 3 * HPL); }

template <typename R, int KZ>
__global__ void __launch_bounds__(TX *BY, 2) k_step(const StepParams<R> p, const int jstep) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sE = reinterpret_cast<R *>(smem_raw);     // [3 planes][3 comps][EY][EX]
    R *sHo = sE + 3 * 3 * EPL;                    // [2][3][HY][HX]  H^{n-1/2}
    R *sH = sHo + 2 * 3 * HPL;                    // [2][3][HY][HX]  H^{n+1/2}

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
    const int nzb = (p.nz + KZ - 1) / KZ;
    const int zb = blockIdx.z % nzb, s = blockIdx.z / nzb;
    const int k0 = zb * KZ, k1 = min(k0 + KZ, p.nz);
    const int n = *p.step + jstep;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml, np2 = 2 * npml;
    const int vol = (int)p.vol, plane = (int)p.plane, pitch = p.pitch;

    const R *__restrict__ E = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    R *__restrict__ En = p.ering + (long long)s * p.ering_stride + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    const R *__restrict__ Hi = ((n & 1) ? p.H2 : p.H) + (long long)s * 3 * p.vol;
    R *__restrict__ Ho = ((n & 1) ? p.H : p.H2) + (long long)s * 3 * p.vol;
    R *__restrict__ P = p.psi + (long long)s * p.psi_stride;
    // slab arrays per axis: [0],[1] H-update memory (buffer A), [2],[3] E-update memory, [4],[5] H (buffer B)
    const int hin = (n & 1) ? 4 : 0, hout = (n & 1) ? 0 : 4;
    R *__restrict__ psx = P;
    R *__restrict__ psy = P + 6 * p.sx;
    R *__restrict__ psz = P + 6 * p.sx + 6 * p.sy;
    const R cH = p.cH;

    // ---- staging of one E plane (tile + full halo) and one H^{n-1/2} plane (tile + low halo)
    auto stage_E = [&](int k, int buf) {
        const bool kin = (k >= 0 && k < p.NZ);
        for (int u = tid; u < 3 * EPL; u += TX * BY) {
            const int c = u / EPL, r = u - c * EPL, ey = r / EX, ex = r - ey * EX;
            const int gi = i0 - 1 + ex, gj = j0 - 1 + ey;
            const bool ok = kin && gi >= 0 && gi < p.NX && gj >= 0 && gj < p.NY;
            const R *src = E + (long long)c * vol + (ok ? k * plane + gj * pitch + gi : 0);
            cp_async_or_zero(sE + (buf * 3 + c) * EPL + r, src, ok);
        }
    };
    auto stage_H = [&](int k, int buf) {
        const bool kin = (k >= 0 && k < nz);
        for (int u = tid; u < 3 * HPL; u += TX * BY) {
            const int c = u / HPL, r = u - c * HPL, hy = r / HX, hx = r - hy * HX;
            const int gi = i0 - 1 + hx, gj = j0 - 1 + hy;
            const bool ok = kin && gi >= 0 && gi < nx && gj >= 0 && gj < ny;
            const R *src = Hi + (long long)c * vol + (ok ? k * plane + gj * pitch + gi : 0);
            cp_async_or_zero(sHo + (buf * 3 + c) * HPL + r, src, ok);
        }
    };

    const int kstart = (k0 > 0) ? k0 - 1 : k0;
    stage_E(kstart, kstart % 3);
    stage_E(kstart + 1, (kstart + 1) % 3);
    stage_H(kstart, kstart % 2);
    cp_async_commit();

    for (int k = kstart; k < k1; ++k) {
        stage_E(k + 2, (k + 2) % 3);        // prefetch for the next iteration
        stage_H(k + 1, (k + 1) % 2);
        cp_async_commit();
        cp_async_wait_1();
        __syncthreads();

        const R *e0 = sE + (k % 3) * 3 * EPL;           // E^n plane k
        const R *e1 = sE + ((k + 1) % 3) * 3 * EPL;     // E^n plane k+1
        const R *ho = sHo + (k % 2) * 3 * HPL;
        R *hn = sH + (k % 2) * 3 * HPL;
        const bool wr = (k >= k0);
        // ---- H^{n+1/2} on tile + low halo
        const int szh = slab_half(k, nz, npml);
        const R ihz = ldg_r(p.az.ih_h + k);
        R bz = 0, az_ = 0;
        if (szh >= 0) { bz = ldg_r(p.az.b_h + k); az_ = ldg_r(p.az.a_h + k); }
        for (int u = tid; u < HPL; u += TX * BY) {
            const int hy = u / HX, hx = u - hy * HX;
            const int gi = i0 - 1 + hx, gj = j0 - 1 + hy;
            R hxn = 0, hyn = 0, hzn = 0;
            if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) {
                const int eo = hy * EX + hx;            // E tile index of (gi, gj)
                const R ex = e0[eo], ey = e0[EPL + eo], ez = e0[2 * EPL + eo];
                const R ihx = ldg_r(p.ax.ih_h + gi), ihy = ldg_r(p.ay.ih_h + gj);
                R dEz_dy = (e0[2 * EPL + eo + EX] - ez) * ihy;
                R dEy_dz = (e1[EPL + eo] - ey) * ihz;
                R dEx_dz = (e1[eo] - ex) * ihz;
                R dEz_dx = (e0[2 * EPL + eo + 1] - ez) * ihx;
                R dEy_dx = (e0[EPL + eo + 1] - ey) * ihx;
                R dEx_dy = (e0[eo + EX] - ex) * ihy;
                const bool own = wr && hx >= 1 && hy >= 1;
                const int sxh = slab_half(gi, nx, npml), syh = slab_half(gj, ny, npml);
                if (syh >= 0) {
                    const R b = ldg_r(p.ay.b_h + gj), a = ldg_r(p.ay.a_h + gj);
                    const int o = (k * np2 + syh) * pitch + gi;
                    const R p0 = b * psy[hin * p.sy + o] + a * dEz_dy;
                    const R p1 = b * psy[(hin + 1) * p.sy + o] + a * dEx_dy;
                    if (own) { psy[hout * p.sy + o] = p0; psy[(hout + 1) * p.sy + o] = p1; }
                    dEz_dy += p0;
                    dEx_dy += p1;
                }
                if (szh >= 0) {
                    const int o = (szh * p.NY + gj) * pitch + gi;
                    const R p0 = bz * psz[hin * p.sz + o] + az_ * dEy_dz;
                    const R p1 = bz * psz[(hin + 1) * p.sz + o] + az_ * dEx_dz;
                    if (own) { psz[hout * p.sz + o] = p0; psz[(hout + 1) * p.sz + o] = p1; }
                    dEy_dz += p0;
                    dEx_dz += p1;
                }
                if (sxh >= 0) {
                    const R b = ldg_r(p.ax.b_h + gi), a = ldg_r(p.ax.a_h + gi);
                    const int o = (k * p.NY + gj) * np2 + sxh;
                    const R p0 = b * psx[hin * p.sx + o] + a * dEz_dx;
                    const R p1 = b * psx[(hin + 1) * p.sx + o] + a * dEy_dx;
                    if (own) { psx[hout * p.sx + o] = p0; psx[(hout + 1) * p.sx + o] = p1; }
                    dEz_dx += p0;
                    dEy_dx += p1;
                }
                hxn = ho[u] - cH * (dEz_dy - dEy_dz);
                hyn = ho[HPL + u] - cH * (dEx_dz - dEz_dx);
                hzn = ho[2 * HPL + u] - cH * (dEy_dx - dEx_dy);
                if (own) {
                    const int idx = k * plane + gj * pitch + gi;
                    Ho[idx] = hxn;
                    Ho[vol + idx] = hyn;
                    Ho[2 * vol + idx] = hzn;
                }
            }
            hn[u] = hxn;
            hn[HPL + u] = hyn;
            hn[2 * HPL + u] = hzn;
        }
        __syncthreads();

        // ---- E^{n+1} on the tile
        if (wr) {
            const R *hm = sH + ((k + 1) % 2) * 3 * HPL;   // H^{n+1/2} plane k-1 (valid when k > 0)
            const int szn = slab_node(k, nz, npml);
            const R ihzn = ldg_r(p.az.ih_n + k);
            R bzn = 0, azn = 0;
            if (szn >= 0) { bzn = ldg_r(p.az.b_n + k); azn = ldg_r(p.az.a_n + k); }
#pragma unroll
            for (int rr = 0; rr < TY / BY; ++rr) {
                const int ly = ty + rr * BY;
                const int gi = i0 + tx, gj = j0 + ly;
                if (gi >= nx || gj >= ny) continue;
                const int h = (ly + 1) * HX + (tx + 1);      // H tile index of (gi, gj)
                const int eo = (ly + 1) * EX + (tx + 1);     // E tile index of (gi, gj)
                const int idx = k * plane + gj * pitch + gi;
                const R hxc = hn[h], hyc = hn[HPL + h], hzc = hn[2 * HPL + h];
                const R ihx = ldg_r(p.ax.ih_n + gi), ihy = ldg_r(p.ay.ih_n + gj);
                const int sxn = slab_node(gi, nx, npml), syn = slab_node(gj, ny, npml);
                if (gj >= 1 && k >= 1) {                     // Ex at (i+1/2, j, k)
                    R dHz_dy = (hzc - hn[2 * HPL + h - HX]) * ihy;
                    R dHy_dz = (hyc - hm[HPL + h]) * ihzn;
                    if (syn >= 0) {
                        R &ps = psy[2 * p.sy + (k * np2 + syn) * pitch + gi];
                        ps = ldg_r(p.ay.b_n + gj) * ps + ldg_r(p.ay.a_n + gj) * dHz_dy;
                        dHz_dy += ps;
                    }
                    if (szn >= 0) {
                        R &ps = psz[2 * p.sz + (szn * p.NY + gj) * pitch + gi];
                        ps = bzn * ps + azn * dHy_dz;
                        dHy_dz += ps;
                    }
                    En[idx] = e0[eo] + ldg_r(p.cE + idx) * (dHz_dy - dHy_dz);
                }
                if (gi >= 1 && k >= 1) {                     // Ey at (i, j+1/2, k)
                    R dHx_dz = (hxc - hm[h]) * ihzn;
                    R dHz_dx = (hzc - hn[2 * HPL + h - 1]) * ihx;
                    if (szn >= 0) {
                        R &ps = psz[3 * p.sz + (szn * p.NY + gj) * pitch + gi];
                        ps = bzn * ps + azn * dHx_dz;
                        dHx_dz += ps;
                    }
                    if (sxn >= 0) {
                        R &ps = psx[2 * p.sx + (k * p.NY + gj) * np2 + sxn];
                        ps = ldg_r(p.ax.b_n + gi) * ps + ldg_r(p.ax.a_n + gi) * dHz_dx;
                        dHz_dx += ps;
                    }
                    En[vol + idx] = e0[EPL + eo] + ldg_r(p.cE + vol + idx) * (dHx_dz - dHz_dx);
                }
                if (gi >= 1 && gj >= 1) {                    // Ez at (i, j, k+1/2)
                    R dHy_dx = (hyc - hn[HPL + h - 1]) * ihx;
                    R dHx_dy = (hxc - hn[h - HX]) * ihy;
                    if (sxn >= 0) {
                        R &ps = psx[3 * p.sx + (k * p.NY + gj) * np2 + sxn];
                        ps = ldg_r(p.ax.b_n + gi) * ps + ldg_r(p.ax.a_n + gi) * dHy_dx;
                        dHy_dx += ps;
                    }
                    if (syn >= 0) {
                        R &ps = psy[3 * p.sy + (k * np2 + syn) * pitch + gi];
                        ps = ldg_r(p.ay.b_n + gj) * ps + ldg_r(p.ay.a_n + gj) * dHx_dy;
                        dHx_dy += ps;
                    }
                    En[2 * vol + idx] = e0[2 * EPL + eo] + ldg_r(p.cE + 2 * vol + idx) * (dHy_dx - dHx_dy);
                }
            }
        }
        __syncthreads();
    }
    cp_async_wait_all();

    // ---- source term E^{n+1} -= dt/eps J'^{n+1/2}: the thread owning a column applies its taps
    if (p.colmap) {
#pragma unroll
        for (int rr = 0; rr < TY / BY; ++rr) {
            const int gi = i0 + tx, gj = j0 + ty + rr * BY;
            if (gi >= nx || gj >= ny) continue;
            const int2 cm = p.colmap[s * p.colmap_stride + gj * pitch + gi];
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
                if (add != 0.0) En[o] += (R)add;
            }
        }
    }
}

template <typename R, int KZ>
void launch_step_kz(const StepParams<R> &p, int S, int jstep, cudaStream_t st) {
    dim3 grid((unsigned)((p.nx + TX - 1) / TX), (unsigned)((p.ny + TY - 1) / TY),
              (unsigned)(((p.nz + KZ - 1) / KZ) * S));
    k_step<R, KZ><<<grid, dim3(TX, BY), fused_smem_bytes(sizeof(R)), st>>>(p, jstep);
}

template <typename R>
cudaError_t launch_fused(const StepParams<R> &p, int S, int jstep, int kz, cudaStream_t st) {
    switch (kz) {
        case 4: launch_step_kz<R, 4>(p, S, jstep, st); break;
        case 8: launch_step_kz<R, 8>(p, S, jstep, st); break;
        case 16: launch_step_kz<R, 16>(p, S, jstep, st); break;
        default: return cudaErrorInvalidValue;
    }
    g_launches++;
    return cudaGetLastError();
}

template <typename R>
cudaError_t prepare_fused() {
    const int sm = (int)fused_smem_bytes(sizeof(R));
    cudaError_t e = cudaFuncSetAttribute(k_step<R, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_step<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

cudaError_t prepare_fused_all() {
    cudaError_t e = prepare_fused<float>();
    if (e == cudaSuccess) e = prepare_fused<double>();
    return e;
}

template cudaError_t launch_fused<float>(const StepParams<float> &, int, int, int, cudaStream_t);
template cudaError_t launch_fused<double>(const StepParams<double> &, int, int, int, cudaStream_t);

}  // namespace csem
