// Early end of forward data runs (Sec. 2: the stepping can stop once the
// frequency-domain field has reached its steady state; the field is checked
// regularly during the run).
#pragma once
#include "csem_internal.cuh"

namespace csem {

// After a chunk of steps: converged when every entry of the running receiver
// transform racc [n] moved by at most tol |racc| since the previous check (never at
// chunk 0).  prev takes racc.  On convergence, or when last is set, fin takes racc
// and state = {1, steps_at}; once state[0] is set later calls change nothing.
cudaError_t launch_es_check(const double2 *racc, double2 *prev, double2 *fin, int n, double tol, int chunk,
                            int last, int steps_at, int *state, cudaStream_t st);

// Runs that keep volumes.  Per frequency f, over every source, component and
// entry of the accumulators acc [S][3][nf][vol]: stats[f] = max |acc| (bit pattern of
// a non-negative float, combined by atomicMax) and stats[nf + f] = 1 if for some entry
// tail.f[f] |acc - prev| > tol max(|acc|, floor_frac stats[2 nf + f]), stats[2 nf + f]
// being the previous check's max (both cleared by the caller, the last kept); prev takes
// acc.  Magnitudes and the comparison in FP32.  tail.f[f]: the remainder of an endless
// run per unit change over the last chunk, for a field that stays as it was.
struct EsTail {
    float f[kMaxFreq];
};
template <typename R>
cudaError_t launch_es_vol_stats(const typename C2<R>::T *acc, typename C2<R>::T *prev, long long vol, int S, int nf,
                                double tol, double floor_frac, const EsTail &tail, unsigned *stats, cudaStream_t st);
// state = {1, steps_at} when chunk >= 1 and no frequency has a moved entry, or when last;
// stats[2 nf + f] takes stats[f] for the next check.
cudaError_t launch_es_vol_decide(unsigned *stats, int nf, int chunk, int last, int steps_at, int *state,
                                 cudaStream_t st);

}  // namespace csem
