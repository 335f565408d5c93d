// Finding kernels for a detector with endcap disks (Sec. 2: barrel layers and
// endcap disks, the event split into eta regions): the DISK instantiations of
// the kernels of kf_find.cuh, compiled apart from the barrel variants.
#include "kf_find.cuh"

namespace kfg {

namespace {
template <int G, int CAP>
cudaError_t prepare_d(int threads, int n_layers, int n_hist, int n_eta, int* blocks_per_sm) {
  return prepare_t<G, CAP, true>(threads, n_layers, n_hist, n_eta, blocks_per_sm);
}
template <int G, int CAP>
cudaError_t launch_main_d(const FindParams& P, int threads, int grid_cap, cudaStream_t st) {
  return launch_main_t<G, CAP, true>(P, threads, grid_cap, st);
}
template <int G, int CAP>
cudaError_t launch_careful_d(const FindParams& P, int grid, cudaStream_t st) {
  return launch_careful_t<G, CAP, true>(P, grid, st);
}
}  // namespace

cudaError_t find_prepare_disk(int lanes, int regcap, int threads, const DevGeom& g, int* blocks_per_sm) {
  KF_FIND_DISPATCH(prepare_d, threads, g.n_layers, g.n_plan, g.n_eta, blocks_per_sm)
}

cudaError_t launch_find_main_disk(const FindParams& P, int lanes, int regcap, int threads, int grid_cap,
                                  cudaStream_t st) {
  const int n = P.s_end - P.s_begin;
  k_seed_fit<true><<<(n + SEED_THREADS - 1) / SEED_THREADS, SEED_THREADS, 0, st>>>(P);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  KF_FIND_DISPATCH(launch_main_d, P, threads, grid_cap, st)
}

cudaError_t launch_find_careful_disk(const FindParams& P, int lanes, int grid, cudaStream_t st) {
  const int regcap = 0;
  KF_FIND_DISPATCH(launch_careful_d, P, grid, st)
}

}  // namespace kfg
