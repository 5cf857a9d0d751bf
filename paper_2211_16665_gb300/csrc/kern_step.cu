// Leap-frog time step of the fictitious-wave Maxwell system (paper Sec. 2, Eq. 4)
// on a stretched Yee grid with unsplit CPML, fused with the on-the-fly damped
// transform of Eq. 6, plus the point operators (receiver sampling with FP64
// transform, source / adjoint-source injection).  One step is three launches:
//   k_h      H^{n-1/2} -> H^{n+1/2} from E^n; also accumulates E^n * w_{k,n}
//            into every frequency's volume (E^n is read here anyway);
//   k_points per source: sample E^n at the receivers and accumulate their FP64
//            transform, then add -dt/eps J'^{n+1/2} at the injection taps;
//   k_e      E^n -> E^{n+1} from curl H^{n+1/2}.
// Threads are laid out flat over the (j, i) plane of the padded lattice and
// march KZ planes along z, keeping the z-neighbour in registers.
#include <atomic>

#include "csem_internal.cuh"

namespace csem {

template <typename R> __device__ __forceinline__ R ldg(const R *p) { return __ldg(p); }

template <typename R>
__device__ __forceinline__ void kahan_add(R &sum, R &c, R x) {
    // compensated summation; the explicit _rn ops keep the compiler from fusing
    R y = x - c;
    R t = sum + y;
    c = (t - sum) - y;
    sum = t;
}
__device__ __forceinline__ void kahan_add(float &sum, float &c, float x) {
    float y = __fsub_rn(x, c);
    float t = __fadd_rn(sum, y);
    c = __fsub_rn(__fsub_rn(t, sum), y);
    sum = t;
}

template <typename R, bool DFT, bool KAHAN>
__global__ void __launch_bounds__(kBlock) k_h(const StepParams<R> p, const int jstep) {
    typedef typename C2<R>::T R2;
    const int t = blockIdx.x * kBlock + threadIdx.x;
    const int j = t / p.pitch;
    const int i = t - j * p.pitch;
    if (j >= p.NY || i >= p.NX) return;
    const int s = blockIdx.z;
    const int k0 = blockIdx.y * p.KZ;
    const int k1 = min(k0 + p.KZ, p.NZ);
    const long long vol = p.vol, plane = p.plane, pitch = p.pitch;
    R *F = p.fields + (long long)s * 6 * vol;
    const R *Ex = F, *Ey = F + vol, *Ez = F + 2 * vol;
    R *Hx = F + 3 * vol, *Hy = F + 4 * vol, *Hz = F + 5 * vol;
    R *P = p.psi + (long long)s * p.psi_stride;
    R *psx = P;                         // 4 x-slab arrays: [0]=Hy,[1]=Hz used here
    R *psy = P + 4 * p.sx;              // 4 y-slab arrays: [0]=Hx,[1]=Hz
    R *psz = P + 4 * p.sx + 4 * p.sy;   // 4 z-slab arrays: [0]=Hx,[1]=Hy
    const int nx = p.nx, ny = p.ny, nz = p.nz, np2 = 2 * p.npml;

    const int sxh = slab_half(i, nx, p.npml);
    const int syh = slab_half(j, ny, p.npml);
    const R ihx = (i < nx) ? ldg(p.ax.ih_h + i) : R(0);
    const R ihy = (j < ny) ? ldg(p.ay.ih_h + j) : R(0);
    R bx = 0, axc = 0, by = 0, ayc = 0;
    if (sxh >= 0) { bx = ldg(p.ax.b_h + i); axc = ldg(p.ax.a_h + i); }
    if (syh >= 0) { by = ldg(p.ay.b_h + j); ayc = ldg(p.ay.a_h + j); }
    const R cH = p.cH;

    R2 wv[kMaxFreq];
    if (DFT) {
        const int n = *p.step + jstep;
        const R2 *w = p.w + (long long)n * p.nf;
#pragma unroll
        for (int f = 0; f < kMaxFreq; ++f)
            if (f < p.nf) wv[f] = w[f];
    }

    long long idx = (long long)k0 * plane + (long long)j * pitch + i;
    R exc = Ex[idx], eyc = Ey[idx];
    for (int k = k0; k < k1; ++k, idx += plane) {
        const R ezc = Ez[idx];
        const bool up = (k + 1 < p.NZ);
        const R exk = up ? Ex[idx + plane] : R(0);
        const R eyk = up ? Ey[idx + plane] : R(0);
        const int szh = slab_half(k, nz, p.npml);
        const R ihz = (k < nz) ? ldg(p.az.ih_h + k) : R(0);
        R bz = 0, azc = 0;
        if (szh >= 0) { bz = ldg(p.az.b_h + k); azc = ldg(p.az.a_h + k); }

        if (j < ny && k < nz) {           // Hx at (i, j+1/2, k+1/2)
            R dEz_dy = (Ez[idx + pitch] - ezc) * ihy;
            R dEy_dz = (eyk - eyc) * ihz;
            if (syh >= 0) {
                R &ps = psy[((long long)k * np2 + syh) * pitch + i];
                ps = by * ps + ayc * dEz_dy;
                dEz_dy += ps;
            }
            if (szh >= 0) {
                R &ps = psz[((long long)szh * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dEy_dz;
                dEy_dz += ps;
            }
            Hx[idx] -= cH * (dEz_dy - dEy_dz);
        }
        if (i < nx && k < nz) {           // Hy at (i+1/2, j, k+1/2)
            R dEx_dz = (exk - exc) * ihz;
            R dEz_dx = (Ez[idx + 1] - ezc) * ihx;
            if (szh >= 0) {
                R &ps = psz[p.sz + ((long long)szh * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dEx_dz;
                dEx_dz += ps;
            }
            if (sxh >= 0) {
                R &ps = psx[((long long)k * p.NY + j) * np2 + sxh];
                ps = bx * ps + axc * dEz_dx;
                dEz_dx += ps;
            }
            Hy[idx] -= cH * (dEx_dz - dEz_dx);
        }
        if (i < nx && j < ny) {           // Hz at (i+1/2, j+1/2, k)
            R dEy_dx = (Ey[idx + 1] - eyc) * ihx;
            R dEx_dy = (Ex[idx + pitch] - exc) * ihy;
            if (sxh >= 0) {
                R &ps = psx[p.sx + ((long long)k * p.NY + j) * np2 + sxh];
                ps = bx * ps + axc * dEy_dx;
                dEy_dx += ps;
            }
            if (syh >= 0) {
                R &ps = psy[p.sy + ((long long)k * np2 + syh) * pitch + i];
                ps = by * ps + ayc * dEx_dy;
                dEx_dy += ps;
            }
            Hz[idx] -= cH * (dEy_dx - dEx_dy);
        }
        if (DFT) {                        // damped transform of E^n (Eq. 6)
            const R e3[3] = {exc, eyc, ezc};
            R2 *A = p.acc + (long long)s * 3 * p.nf * vol + idx;
            R2 *Cm = KAHAN ? p.comp + (long long)s * 3 * p.nf * vol + idx : nullptr;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int f = 0; f < kMaxFreq; ++f) {
                    if (f >= p.nf) break;
                    const long long o = (long long)(c * p.nf + f) * vol;
                    R2 a = A[o];
                    if (KAHAN) {
                        R2 cc = Cm[o];
                        kahan_add(a.x, cc.x, e3[c] * wv[f].x);
                        kahan_add(a.y, cc.y, e3[c] * wv[f].y);
                        Cm[o] = cc;
                    } else {
                        a.x += e3[c] * wv[f].x;
                        a.y += e3[c] * wv[f].y;
                    }
                    A[o] = a;
                }
            }
        }
        exc = exk;
        eyc = eyk;
    }
}

template <typename R>
__global__ void __launch_bounds__(kBlock) k_e(const StepParams<R> p) {
    const int t = blockIdx.x * kBlock + threadIdx.x;
    const int j = t / p.pitch;
    const int i = t - j * p.pitch;
    if (j >= p.NY || i >= p.NX) return;
    const int s = blockIdx.z;
    const int k0 = blockIdx.y * p.KZ;
    const int k1 = min(k0 + p.KZ, p.NZ);
    const long long vol = p.vol, plane = p.plane, pitch = p.pitch;
    R *F = p.fields + (long long)s * 6 * vol;
    R *Ex = F, *Ey = F + vol, *Ez = F + 2 * vol;
    const R *Hx = F + 3 * vol, *Hy = F + 4 * vol, *Hz = F + 5 * vol;
    const R *cEx = p.cE, *cEy = p.cE + vol, *cEz = p.cE + 2 * vol;
    R *P = p.psi + (long long)s * p.psi_stride;
    R *psx = P;                         // [2]=Ey(dHz/dx) [3]=Ez(dHy/dx)
    R *psy = P + 4 * p.sx;              // [2]=Ex(dHz/dy) [3]=Ez(dHx/dy)
    R *psz = P + 4 * p.sx + 4 * p.sy;   // [2]=Ex(dHy/dz) [3]=Ey(dHx/dz)
    const int nx = p.nx, ny = p.ny, nz = p.nz, np2 = 2 * p.npml;

    const int sxn = slab_node(i, nx, p.npml);
    const int syn = slab_node(j, ny, p.npml);
    const R ihx = ldg(p.ax.ih_n + i);
    const R ihy = ldg(p.ay.ih_n + j);
    R bx = 0, axc = 0, by = 0, ayc = 0;
    if (sxn >= 0) { bx = ldg(p.ax.b_n + i); axc = ldg(p.ax.a_n + i); }
    if (syn >= 0) { by = ldg(p.ay.b_n + j); ayc = ldg(p.ay.a_n + j); }
    const bool ix_in = (i >= 1 && i < nx), jy_in = (j >= 1 && j < ny);

    long long idx = (long long)k0 * plane + (long long)j * pitch + i;
    R hxm = (k0 > 0) ? Hx[idx - plane] : R(0);
    R hym = (k0 > 0) ? Hy[idx - plane] : R(0);
    for (int k = k0; k < k1; ++k, idx += plane) {
        const R hxc = Hx[idx], hyc = Hy[idx], hzc = Hz[idx];
        const int szn = slab_node(k, nz, p.npml);
        const R ihz = ldg(p.az.ih_n + k);
        R bz = 0, azc = 0;
        if (szn >= 0) { bz = ldg(p.az.b_n + k); azc = ldg(p.az.a_n + k); }
        const bool kz_in = (k >= 1 && k < nz);

        if (i < nx && jy_in && kz_in) {   // Ex at (i+1/2, j, k)
            R dHz_dy = (hzc - Hz[idx - pitch]) * ihy;
            R dHy_dz = (hyc - hym) * ihz;
            if (syn >= 0) {
                R &ps = psy[2 * p.sy + ((long long)k * np2 + syn) * pitch + i];
                ps = by * ps + ayc * dHz_dy;
                dHz_dy += ps;
            }
            if (szn >= 0) {
                R &ps = psz[2 * p.sz + ((long long)szn * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dHy_dz;
                dHy_dz += ps;
            }
            Ex[idx] += ldg(cEx + idx) * (dHz_dy - dHy_dz);
        }
        if (j < ny && ix_in && kz_in) {   // Ey at (i, j+1/2, k)
            R dHx_dz = (hxc - hxm) * ihz;
            R dHz_dx = (hzc - Hz[idx - 1]) * ihx;
            if (szn >= 0) {
                R &ps = psz[3 * p.sz + ((long long)szn * p.NY + j) * pitch + i];
                ps = bz * ps + azc * dHx_dz;
                dHx_dz += ps;
            }
            if (sxn >= 0) {
                R &ps = psx[2 * p.sx + ((long long)k * p.NY + j) * np2 + sxn];
                ps = bx * ps + axc * dHz_dx;
                dHz_dx += ps;
            }
            Ey[idx] += ldg(cEy + idx) * (dHx_dz - dHz_dx);
        }
        if (k < nz && ix_in && jy_in) {   // Ez at (i, j, k+1/2)
            R dHy_dx = (hyc - Hy[idx - 1]) * ihx;
            R dHx_dy = (hxc - Hx[idx - pitch]) * ihy;
            if (sxn >= 0) {
                R &ps = psx[3 * p.sx + ((long long)k * p.NY + j) * np2 + sxn];
                ps = bx * ps + axc * dHy_dx;
                dHy_dx += ps;
            }
            if (syn >= 0) {
                R &ps = psy[3 * p.sy + ((long long)k * np2 + syn) * pitch + i];
                ps = by * ps + ayc * dHx_dy;
                dHx_dy += ps;
            }
            Ez[idx] += ldg(cEz + idx) * (dHy_dx - dHx_dy);
        }
        hxm = hxc;
        hym = hyc;
    }
}

// One block per source: receivers first (they read E^n), then injection
// (it writes E^n before the E update).  Sources own disjoint fields.
template <typename R>
__global__ void __launch_bounds__(kBlock) k_points(const PointParams<R> q, const int jstep) {
    const int s = blockIdx.x;
    const int n = *q.step + jstep;
    R *F = q.fields + (long long)s * 6 * q.vol;
    for (int r = threadIdx.x; r < q.n_rec; r += blockDim.x) {
        double v = 0.0;
        const Tap *tp = q.rtaps + (long long)r * 8;
#pragma unroll
        for (int m = 0; m < 8; ++m) v += tp[m].w * (double)F[(long long)tp[m].comp * q.vol + tp[m].idx];
        double2 *a = q.racc + ((long long)s * q.n_rec + r) * q.nf;
        const double2 *w = q.w64 + (long long)n * q.nf;
        for (int f = 0; f < q.nf; ++f) {
            double2 t = a[f];
            t.x += v * w[f].x;
            t.y += v * w[f].y;
            a[f] = t;
        }
        if (q.trace) q.trace[((long long)s * q.n_rec + r) * q.nt + n] = v;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < q.n_itaps; m += blockDim.x) {
        const Tap tp = q.itaps[(long long)s * q.itap_stride + m];
        const double *cf = q.coef + ((long long)s * q.n_emit + tp.emit) * q.J;
        const double *T = q.T + (long long)n * q.J;
        double amp = 0.0;
        for (int jj = 0; jj < q.J; ++jj) amp += cf[jj] * T[jj];
        const long long o = (long long)tp.comp * q.vol + tp.idx;
        const double add = -(double)q.cE[o] * tp.w * amp;
        if (add != 0.0) atomicAdd(F + o, (R)add);
    }
}

__global__ void k_advance(int *step, int by) { *step += by; }

std::atomic<long long> g_launches{0};

template <typename R>
cudaError_t launch_step(const StepParams<R> &p, const PointParams<R> &q, int S, int jstep, bool dft, bool kahan,
                        cudaStream_t st, int which) {
    const long long plane_threads = (long long)p.NY * p.pitch;
    dim3 grid((unsigned)((plane_threads + kBlock - 1) / kBlock), (unsigned)((p.NZ + p.KZ - 1) / p.KZ), (unsigned)S);
    if (which & 1) {
        if (!dft) k_h<R, false, false><<<grid, kBlock, 0, st>>>(p, jstep);
        else if (kahan) k_h<R, true, true><<<grid, kBlock, 0, st>>>(p, jstep);
        else k_h<R, true, false><<<grid, kBlock, 0, st>>>(p, jstep);
        g_launches++;
    }
    if ((which & 2) && (q.n_rec > 0 || q.n_itaps > 0)) {
        k_points<R><<<S, kBlock, 0, st>>>(q, jstep);
        g_launches++;
    }
    if (which & 4) {
        k_e<R><<<grid, kBlock, 0, st>>>(p);
        g_launches++;
    }
    return cudaGetLastError();
}

cudaError_t launch_advance(int *step, int by, cudaStream_t st) {
    k_advance<<<1, 1, 0, st>>>(step, by);
    g_launches++;
    return cudaGetLastError();
}

template cudaError_t launch_step<float>(const StepParams<float> &, const PointParams<float> &, int, int, bool, bool,
                                        cudaStream_t, int);
template cudaError_t launch_step<double>(const StepParams<double> &, const PointParams<double> &, int, int, bool,
                                         bool, cudaStream_t, int);

}  // namespace csem
