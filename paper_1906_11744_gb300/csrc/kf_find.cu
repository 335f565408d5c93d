// Finding entry points (Sec. 2): the barrel variants of the kernels of
// kf_find.cuh, the seed order, and the dispatch to the disk variants
// (kf_find_disk.cu) for a detector with endcap disks.
#include "kf_find.cuh"

namespace kfg {

namespace {

// Order in which the finding takes the seeds of each event: by polar angle
// theta (counting sort into SEED_THETA_BINS bins, one block per event).  The
// seeds of a warp then cross about as many layers before they leave the
// barrel, which keeps its groups busy for the same number of iterations; the
// result of a seed does not depend on the order.
constexpr int THETA_BINS = SEED_THETA_BINS;
__global__ void __launch_bounds__(1024) k_seed_order(const float* theta, const int* seed_off, int* order) {
  __shared__ unsigned cnt[THETA_BINS];
  __shared__ unsigned sh[33];
  const int s0 = seed_off[blockIdx.x], s1 = seed_off[blockIdx.x + 1];
  for (int k = threadIdx.x; k < THETA_BINS; k += blockDim.x) cnt[k] = 0u;
  __syncthreads();
  auto bin_of = [&](int s) { return seed_theta_bin(theta[s]); };
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) atomicAdd(&cnt[bin_of(s)], 1u);
  __syncthreads();
  // exclusive scan of the THETA_BINS counts (one per thread)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned v = threadIdx.x < THETA_BINS ? cnt[threadIdx.x] : 0u;
  unsigned incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
    const unsigned w = lane < nw ? sh[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) sh[lane] = wi - w;
  }
  __syncthreads();
  if (threadIdx.x < THETA_BINS) cnt[threadIdx.x] = sh[warp] + incl - v;
  __syncthreads();
  for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) order[s0 + atomicAdd(&cnt[bin_of(s)], 1u)] = s;
}

}  // namespace

cudaError_t launch_seed_order(const float* theta, const int* seed_off, int n_events, int* order, cudaStream_t st) {
  if (n_events <= 0) return cudaSuccess;
  k_seed_order<<<n_events, 1024, 0, st>>>(theta, seed_off, order);
  return cudaGetLastError();
}

size_t find_smem_bytes(int threads, int n_layers, int n_eta) {
  return smem_edges(n_layers, n_eta) + (size_t)(threads / 32) * smem_per_warp(KF_MAX_CANDS, false, n_layers);
}

bool find_lanes_supported(int lanes) {
  return lanes == 4 || lanes == 6 || lanes == 8 || lanes == 10 || lanes == 12 || lanes == 16;
}

namespace {
template <int G, int CAP>
cudaError_t prepare_b(int threads, int n_layers, int n_eta, int* blocks_per_sm) {
  return prepare_t<G, CAP, false>(threads, n_layers, n_layers, n_eta, blocks_per_sm);
}
template <int G, int CAP>
cudaError_t launch_main_b(const FindParams& P, int threads, int grid_cap, cudaStream_t st) {
  return launch_main_t<G, CAP, false>(P, threads, grid_cap, st);
}
template <int G, int CAP>
cudaError_t launch_careful_b(const FindParams& P, int grid, cudaStream_t st) {
  return launch_careful_t<G, CAP, false>(P, grid, st);
}
}  // namespace

cudaError_t find_prepare(int lanes, int regcap, int threads, const DevGeom& g, int* blocks_per_sm) {
  if (g.n_disks > 0) return find_prepare_disk(lanes, regcap, threads, g, blocks_per_sm);
  KF_FIND_DISPATCH(prepare_b, threads, g.n_layers, g.n_eta, blocks_per_sm)
}

cudaError_t launch_find_main(const FindParams& P, int lanes, int regcap, int threads, int grid_cap,
                             cudaStream_t st) {
  if (P.s_end <= P.s_begin) return cudaSuccess;
  if (P.g.n_disks > 0) return launch_find_main_disk(P, lanes, regcap, threads, grid_cap, st);
  const int n = P.s_end - P.s_begin;
  k_seed_fit<false><<<(n + SEED_THREADS - 1) / SEED_THREADS, SEED_THREADS, 0, st>>>(P);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  KF_FIND_DISPATCH(launch_main_b, P, threads, grid_cap, st)
}

cudaError_t launch_find_careful(const FindParams& P, int lanes, int grid, cudaStream_t st) {
  if (P.s_end <= P.s_begin) return cudaSuccess;
  if (P.g.n_disks > 0) return launch_find_careful_disk(P, lanes, grid, st);
  const int regcap = 0;
  KF_FIND_DISPATCH(launch_careful_b, P, grid, st)
}

}  // namespace kfg
