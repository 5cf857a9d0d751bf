// FP32 H and E step kernels fed by the tensor-memory-access engine.
//
// A block owns TY rows (j0 .. j0+TY-1) of full lattice rows (pitch entries) and
// marches the z planes of one chunk [k0, k1).  Every plane it needs is brought
// into shared memory by one thread with cp.async.bulk row copies completing on
// the mbarrier of a three-deep ring of stages, so all rows of a plane and of
// the next one are in flight at once; the other threads compute from shared
// memory and store their results with coalesced row writes.  Waits on the
// barriers are bounded (about a second): a block whose wait gives up leaves the
// plane loop with all its threads together, raises the staged-kernel bit of
// *err, waits (bounded) for every copy it issued and returns.  Same arithmetic,
// per entry, as the other step kernels.
//
//   k_h_tma stage (plane k): E rows j0 .. j0+TY (3 components), H^{n-1/2} rows
//           j0 .. j0+TY-1 (3 components); plane k also reads stage k+1's E.
//   k_e_tma stage (plane k): H^{n+1/2} rows j0-1 .. j0+TY-1, E^n and dt/eps rows
//           j0 .. j0+TY-1 (3 components each); plane k also reads H of stage k-1.
#include "csem_internal.cuh"

namespace csem {

namespace {

__device__ __forceinline__ uint32_t s_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t *b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_u32(b)) : "memory");
}
__device__ __forceinline__ void bar_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void bar_expect(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_row(float *dst, const float *src, uint32_t bytes, uint64_t *b) {
    uint64_t g;
    asm volatile("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     s_u32(dst)),
                 "l"(g), "r"(bytes), "r"(s_u32(b))
                 : "memory");
}
}  // namespace

template <int TY>
__global__ void __launch_bounds__(kBlock, 1) k_h_tma(const StepParams<float> p, const int jstep, const int KZ,
                                                     int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[3];
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int P = p.pitch, vol = (int)p.vol, plane = (int)p.plane;
    constexpr int RE = 3 * (TY + 1), RS = RE + 3 * TY;   // rows per stage: E then H
    const int j0 = blockIdx.x * TY;
    const int k0 = blockIdx.y * KZ, k1 = min(k0 + KZ, p.nz);
    const int s = blockIdx.z;
    const int n = *p.step + jstep;
    const float *E = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    float *H = p.H + (long long)s * 3 * vol;
    float *Pp = p.psi + (long long)s * p.psi_stride;
    float *psx = Pp, *psy = Pp + 6 * p.sx, *psz = Pp + 6 * p.sx + 6 * p.sy;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml, np2 = 2 * npml;
    const uint32_t rowb = (uint32_t)P * sizeof(float);

    // stage b holds plane k: E rows j0..j0+TY (rows >= NY skipped), H rows j0..j0+TY-1 (rows >= ny skipped)
    auto issue = [&](int k, bool with_h) {
        const int b = k % 3;
        float *st = sm + (size_t)b * RS * P;
        uint32_t bytes = (k == k0) ? (uint32_t)p.fault_tx : 0u;
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r <= TY; ++r) if (j0 + r < p.NY) bytes += rowb;
        if (with_h)
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < TY; ++r) if (j0 + r < ny) bytes += rowb;
        bar_expect(&bar[b], bytes);
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r <= TY; ++r)
                if (j0 + r < p.NY)
                    bulk_row(st + (c * (TY + 1) + r) * P, E + c * vol + k * plane + (j0 + r) * P, rowb, &bar[b]);
        if (with_h)
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < TY; ++r)
                    if (j0 + r < ny)
                        bulk_row(st + (RE + c * TY + r) * P, H + c * vol + k * plane + (j0 + r) * P, rowb, &bar[b]);
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) bar_init(&bar[b]);
        bar_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        issue(k0, true);
        issue(k0 + 1, k0 + 1 < k1);            // plane k1 <= nz exists: E only
    }
    int hi = k0 + 1;                           // highest plane issued
    uint32_t ph = 0;
    const float cH = p.cH;
    bool ok = mbar_wait_bounded(&bar[k0 % 3], 0);
    ph ^= 1u << (k0 % 3);
    int k = k0;
    for (; k < k1; ++k) {
        const int b = k % 3, b1 = (k + 1) % 3;
        if (ok) ok = mbar_wait_bounded(&bar[b1], (ph >> b1) & 1);   // plane k+1 (plane k is already in)
        ph ^= 1u << b1;
        // every thread has finished plane k-1 (its stage is free); a give-up ends the loop for all
        if (__syncthreads_or(!ok)) break;
        if (k + 2 <= k1) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(k + 2, k + 2 < k1);       // into the stage plane k-1 used
            }
            hi = k + 2;
        }
        const float *st = sm + (size_t)b * RS * P, *st1 = sm + (size_t)b1 * RS * P;
        const int szh = slab_half(k, nz, npml);
        const float ihz = __ldg(p.az.ih_h + k);
        float bz = 0.f, az = 0.f;
        if (szh >= 0) { bz = __ldg(p.az.b_h + k); az = __ldg(p.az.a_h + k); }
        for (int u = threadIdx.x; u < TY * P; u += blockDim.x) {
            const int r = u / P, i = u - r * P, j = j0 + r;
            if (i >= nx || j >= ny) continue;
            const float *ex = st + r * P, *ey = st + ((TY + 1) + r) * P, *ez = st + (2 * (TY + 1) + r) * P;
            const float exc = ex[i], eyc = ey[i], ezc = ez[i];
            const float ihx = __ldg(p.ax.ih_h + i), ihy = __ldg(p.ay.ih_h + j);
            float dEz_dy = (ez[i + P] - ezc) * ihy;
            float dEy_dz = (st1[((TY + 1) + r) * P + i] - eyc) * ihz;
            float dEx_dz = (st1[r * P + i] - exc) * ihz;
            float dEz_dx = (ez[i + 1] - ezc) * ihx;
            float dEy_dx = (ey[i + 1] - eyc) * ihx;
            float dEx_dy = (ex[i + P] - exc) * ihy;
            const int syh = slab_half(j, ny, npml), sxh = slab_half(i, nx, npml);
            if (syh >= 0) {
                const float by = __ldg(p.ay.b_h + j), ay = __ldg(p.ay.a_h + j);
                const int o = (k * np2 + syh) * P + i;
                float &p0 = psy[o], &p1 = psy[p.sy + o];
                p0 = by * p0 + ay * dEz_dy; dEz_dy += p0;
                p1 = by * p1 + ay * dEx_dy; dEx_dy += p1;
            }
            if (szh >= 0) {
                const int o = (szh * p.NY + j) * P + i;
                float &p0 = psz[o], &p1 = psz[p.sz + o];
                p0 = bz * p0 + az * dEy_dz; dEy_dz += p0;
                p1 = bz * p1 + az * dEx_dz; dEx_dz += p1;
            }
            if (sxh >= 0) {
                const float bx = __ldg(p.ax.b_h + i), ax = __ldg(p.ax.a_h + i);
                const int o = (k * p.NY + j) * np2 + sxh;
                float &p0 = psx[o], &p1 = psx[p.sx + o];
                p0 = bx * p0 + ax * dEz_dx; dEz_dx += p0;
                p1 = bx * p1 + ax * dEy_dx; dEy_dx += p1;
            }
            const float *hs = st + RE * P + r * P;
            const int idx = k * plane + j * P + i;
            H[idx] = hs[i] - cH * (dEz_dy - dEy_dz);
            H[vol + idx] = hs[TY * P + i] - cH * (dEx_dz - dEz_dx);
            H[2 * vol + idx] = hs[2 * TY * P + i] - cH * (dEy_dx - dEx_dy);
        }
    }
    if (k < k1) {                              // gave up: report, let the issued copies land
        if (threadIdx.x == 0) {
            atomicOr(err, kErrStagedWait);
            for (int m = k; m <= hi; ++m) mbar_wait_bounded(&bar[m % 3], (uint32_t)(((m - k0) / 3) & 1));
        }
        __syncthreads();
    }
}

template <int TY>
__global__ void __launch_bounds__(kBlock, 1) k_e_tma(const StepParams<float> p, const int jstep, const int KZ,
                                                     int *err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[3];
    float *sm = reinterpret_cast<float *>(smem_raw);
    const int P = p.pitch, vol = (int)p.vol, plane = (int)p.plane;
    constexpr int RH = 3 * (TY + 1), RS = RH + 6 * TY;   // rows per stage: H, then E^n, then dt/eps
    const int j0 = blockIdx.x * TY;
    const int k0 = blockIdx.y * KZ, k1 = min(k0 + KZ, p.nz);
    const int s = blockIdx.z;
    const int n = *p.step + jstep;
    const float *Eo = p.ering + (long long)s * p.ering_stride + (long long)(n % p.nslot) * 3 * p.vol;
    float *En = p.ering + (long long)s * p.ering_stride + (long long)((n + 1) % p.nslot) * 3 * p.vol;
    const float *H = p.H + (long long)s * 3 * vol;
    float *Pp = p.psi + (long long)s * p.psi_stride;
    float *psx = Pp, *psy = Pp + 6 * p.sx, *psz = Pp + 6 * p.sx + 6 * p.sy;
    const int nx = p.nx, ny = p.ny, nz = p.nz, npml = p.npml, np2 = 2 * npml;
    const uint32_t rowb = (uint32_t)P * sizeof(float);

    // stage of plane k: H rows j0-1 .. j0+TY-1 (rows < 0 skipped), then E^n and dt/eps rows j0 .. j0+TY-1
    const int kf = (k0 > 0) ? k0 - 1 : k0;     // first plane issued
    auto issue = [&](int k, bool h_only) {
        const int b = ((k % 3) + 3) % 3;
        float *st = sm + (size_t)b * RS * P;
        uint32_t bytes = (k == kf) ? (uint32_t)p.fault_tx : 0u;
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r <= TY; ++r) if (j0 - 1 + r >= 0 && j0 - 1 + r < ny) bytes += rowb;
        if (!h_only)
            for (int c = 0; c < 6; ++c)
                for (int r = 0; r < TY; ++r) if (j0 + r < ny) bytes += rowb;
        bar_expect(&bar[b], bytes);
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r <= TY; ++r) {
                const int j = j0 - 1 + r;
                if (j >= 0 && j < ny)
                    bulk_row(st + (c * (TY + 1) + r) * P, H + c * vol + k * plane + j * P, rowb, &bar[b]);
            }
        if (!h_only)
            for (int c = 0; c < 3; ++c)
                for (int r = 0; r < TY; ++r)
                    if (j0 + r < ny) {
                        const int o = k * plane + (j0 + r) * P;
                        bulk_row(st + (RH + c * TY + r) * P, Eo + c * vol + o, rowb, &bar[b]);
                        bulk_row(st + (RH + 3 * TY + c * TY + r) * P, p.cE + c * vol + o, rowb, &bar[b]);
                    }
    };

    if (threadIdx.x == 0) {
        for (int b = 0; b < 3; ++b) bar_init(&bar[b]);
        bar_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (k0 > 0) issue(k0 - 1, true);
        issue(k0, false);
    }
    int hi = k0;                               // highest plane issued
    uint32_t ph = 0;
    bool ok = true;
    int k = k0;
    for (; k < k1; ++k) {
        const int b = k % 3, bm = (k + 2) % 3;  // bm: stage of plane k-1
        if (k == k0 && k0 > 0) {
            ok = mbar_wait_bounded(&bar[bm], (ph >> bm) & 1);
            ph ^= 1u << bm;
        }
        if (ok) ok = mbar_wait_bounded(&bar[b], (ph >> b) & 1);
        ph ^= 1u << b;
        // every thread has finished plane k-1 (the stage of plane k-2 is free); a give-up ends
        // the loop for all
        if (__syncthreads_or(!ok)) break;
        if (k + 1 < k1) {
            if (threadIdx.x == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(k + 1, false);            // into the stage plane k-2 used
            }
            hi = k + 1;
        }
        const float *st = sm + (size_t)b * RS * P, *sm1 = sm + (size_t)bm * RS * P;
        const int szn = slab_node(k, nz, npml);
        const float ihz = __ldg(p.az.ih_n + k);
        float bz = 0.f, az = 0.f;
        if (szn >= 0) { bz = __ldg(p.az.b_n + k); az = __ldg(p.az.a_n + k); }
        const bool kin = (k >= 1);
        for (int u = threadIdx.x; u < TY * P; u += blockDim.x) {
            const int r = u / P, i = u - r * P, j = j0 + r;
            if (i >= nx || j >= ny) continue;
            const float *hx = st + (r + 1) * P, *hy = st + ((TY + 1) + r + 1) * P, *hz = st + (2 * (TY + 1) + r + 1) * P;
            const float hxc = hx[i], hyc = hy[i], hzc = hz[i];
            const float ihx = __ldg(p.ax.ih_n + i), ihy = __ldg(p.ay.ih_n + j);
            const int sxn = slab_node(i, nx, npml), syn = slab_node(j, ny, npml);
            const int idx = k * plane + j * P + i;
            const float *eo = st + (RH + r) * P, *ce = st + (RH + 3 * TY + r) * P;
            if (j >= 1 && kin) {                                      // Ex
                float dHz_dy = (hzc - hz[i - P]) * ihy;
                float dHy_dz = (hyc - sm1[((TY + 1) + r + 1) * P + i]) * ihz;
                if (syn >= 0) {
                    float &ps = psy[2 * p.sy + (k * np2 + syn) * P + i];
                    ps = __ldg(p.ay.b_n + j) * ps + __ldg(p.ay.a_n + j) * dHz_dy;
                    dHz_dy += ps;
                }
                if (szn >= 0) {
                    float &ps = psz[2 * p.sz + (szn * p.NY + j) * P + i];
                    ps = bz * ps + az * dHy_dz;
                    dHy_dz += ps;
                }
                En[idx] = eo[i] + ce[i] * (dHz_dy - dHy_dz);
            }
            if (i >= 1 && kin) {                                      // Ey
                float dHx_dz = (hxc - sm1[(r + 1) * P + i]) * ihz;
                float dHz_dx = (hzc - hz[i - 1]) * ihx;
                if (szn >= 0) {
                    float &ps = psz[3 * p.sz + (szn * p.NY + j) * P + i];
                    ps = bz * ps + az * dHx_dz;
                    dHx_dz += ps;
                }
                if (sxn >= 0) {
                    float &ps = psx[2 * p.sx + (k * p.NY + j) * np2 + sxn];
                    ps = __ldg(p.ax.b_n + i) * ps + __ldg(p.ax.a_n + i) * dHz_dx;
                    dHz_dx += ps;
                }
                En[vol + idx] = eo[TY * P + i] + ce[TY * P + i] * (dHx_dz - dHz_dx);
            }
            if (i >= 1 && j >= 1) {                                   // Ez
                float dHy_dx = (hyc - hy[i - 1]) * ihx;
                float dHx_dy = (hxc - hx[i - P]) * ihy;
                if (sxn >= 0) {
                    float &ps = psx[3 * p.sx + (k * p.NY + j) * np2 + sxn];
                    ps = __ldg(p.ax.b_n + i) * ps + __ldg(p.ax.a_n + i) * dHy_dx;
                    dHy_dx += ps;
                }
                if (syn >= 0) {
                    float &ps = psy[3 * p.sy + (k * np2 + syn) * P + i];
                    ps = __ldg(p.ay.b_n + j) * ps + __ldg(p.ay.a_n + j) * dHx_dy;
                    dHx_dy += ps;
                }
                En[2 * vol + idx] = eo[2 * TY * P + i] + ce[2 * TY * P + i] * (dHy_dx - dHx_dy);
            }
        }
    }
    if (k < k1) {                              // gave up: report, let the issued copies land
        if (threadIdx.x == 0) {
            atomicOr(err, kErrStagedWait);
            for (int m = (k == k0) ? kf : k; m <= hi; ++m) mbar_wait_bounded(&bar[m % 3], (uint32_t)(((m - kf) / 3) & 1));
        }
        __syncthreads();
        return;
    }
    // source term E^{n+1} -= dt/eps J'^{n+1/2}: each column of the tile is handled by one thread
    if (p.colmap) {
        for (int u = threadIdx.x; u < TY * P; u += blockDim.x) {
            const int r = u / P, i = u - r * P, j = j0 + r;
            if (i >= nx || j >= ny) continue;
            const int2 cm = p.colmap[s * p.colmap_stride + j * P + i];
            for (int q = cm.x; q < cm.x + cm.y; ++q) {
                const Tap tp = p.itaps[(long long)s * p.itap_stride + q];
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

size_t tma_smem_bytes(bool h, int ty, int pitch) {
    const int rows = h ? (3 * (ty + 1) + 3 * ty) : (3 * (ty + 1) + 6 * ty);
    return (size_t)3 * rows * pitch * sizeof(float);
}

// Largest TY (1, 2, 4) whose staged planes fit the per-block shared memory limit, 0 if none.
int tma_max_rows(int pitch) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int best = 0;
    for (int ty : {1, 2, 4})
        if ((int)tma_smem_bytes(false, ty, pitch) + 1024 <= optin) best = ty;
    return best;
}

// Lets every staged kernel use up to the device's opt-in shared memory per block.
cudaError_t prepare_tma() {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int lim = optin - 1024;                 // room for the kernels' static barrier words
    cudaError_t e = cudaFuncSetAttribute(k_h_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_h_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_h_tma<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_e_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_e_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_e_tma<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    return e;
}

cudaError_t launch_field_tma(const StepParams<float> &p, int S, int jstep, cudaStream_t st, bool h, int kz, int ty,
                             int *err) {
    dim3 grid((unsigned)((p.ny + ty - 1) / ty), (unsigned)((p.nz + kz - 1) / kz), (unsigned)S);
    const size_t sm = tma_smem_bytes(h, ty, p.pitch);
    switch (ty) {
        case 1: if (h) k_h_tma<1><<<grid, kBlock, sm, st>>>(p, jstep, kz, err); else k_e_tma<1><<<grid, kBlock, sm, st>>>(p, jstep, kz, err); break;
        case 2: if (h) k_h_tma<2><<<grid, kBlock, sm, st>>>(p, jstep, kz, err); else k_e_tma<2><<<grid, kBlock, sm, st>>>(p, jstep, kz, err); break;
        case 4: if (h) k_h_tma<4><<<grid, kBlock, sm, st>>>(p, jstep, kz, err); else k_e_tma<4><<<grid, kBlock, sm, st>>>(p, jstep, kz, err); break;
        default: return cudaErrorInvalidValue;
    }
    g_launches++;
    return cudaGetLastError();
}

}  // namespace csem
