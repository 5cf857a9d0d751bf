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
// entry of the accumulators acc [S][3][nf][vol]: stats[f] = max |acc| and
// stats[nf + f] = max |acc - prev| (bit patterns of non-negative floats, combined by
// atomicMax, cleared by the caller); prev takes acc.
template <typename R>
cudaError_t launch_es_vol_stats(const typename C2<R>::T *acc, typename C2<R>::T *prev, long long vol, int S, int nf,
                                unsigned *stats, cudaStream_t st);
// state = {1, steps_at} when chunk >= 1 and stats[nf + f] <= tol stats[f] for every f, or when last.
cudaError_t launch_es_vol_decide(const unsigned *stats, int nf, double tol, int chunk, int last, int steps_at,
                                 int *state, cudaStream_t st);

}  // namespace csem
