// Fourth-order staggered stepping on the non-uniform grid (Sec. 2: the paper's
// engine uses high-order differences over the non-uniform grid and prints no
// coefficients).  Per axis of n cells:
//   wh[p][0..3]  derivative at the half node p from the nodes p-1 .. p+2,
//   wn[q][0..3]  derivative at the node q from the half nodes q-2 .. q+1,
// each the derivative of the cubic through its four points (exact for cubics);
// the first and last half node and the nodes 1 and n-1 keep the two-point
// difference (weights 0, -1/h, 1/h, 0).  The CPML memory is kept as 12 volume
// arrays per source ([S][12][vol], psi_stride = 12 vol), in the order
//   Hx(dEz/dy) Hx(dEy/dz) Hy(dEx/dz) Hy(dEz/dx) Hz(dEy/dx) Hz(dEx/dy)
//   Ex(dHz/dy) Ex(dHy/dz) Ey(dHx/dz) Ey(dHz/dx) Ez(dHy/dx) Ez(dHx/dy).
#pragma once
#include "csem_internal.cuh"

namespace csem {

template <typename R>
struct HoTab {
    const R *wxh, *wxn, *wyh, *wyn, *wzh, *wzn;   // [n][4] and [n+1][4] per axis
};

// which: bit 0 = H half-step, bit 2 = E step with the source injection of p.  FP32 halves whose
// LEAN flag is set run the lean kernels (KZ planes per thread, MB resident 128-thread blocks).
template <typename R>
cudaError_t launch_ho(const StepParams<R> &p, const HoTab<R> &w, int S, int jstep, cudaStream_t st, int which);
// lean FP32 kernels: nx even, kz in {2, 4, 8}, mb in {4, 6, 8}; need the masked dt/eps and the padded tables
cudaError_t launch_ho4(const StepParams<float> &p, const HoTab<float> &w, int S, int jstep, cudaStream_t st, bool h,
                       int kz, int mb);
bool ho4_supported(int kz, int mb);

}  // namespace csem
