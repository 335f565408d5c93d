// Hit binning: counting sort of every hit into its (event, layer, eta bin,
// phi bin) cell, so that a search window is a few contiguous ranges of the
// binned array (the GPU form of the paper's per-layer hit search windows,
// Sec. 3).  The grid is n_eta bins in eta = asinh(z/R_layer) over
// [-asinh(z_max/R), +asinh(z_max/R)] (as z edges per layer) times n_phi bins
// in phi = atan2(y, x).
//
//   1. k_bin_count   : key and rank of each hit (atomic count per cell);
//   2. exclusive scan of the counts into global offsets (three passes);
//   3. k_bin_scatter : hit -> binned array at offset[key] + rank.
#include "kf_internal.h"

namespace kfg {

namespace {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_PER_THREAD = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_PER_THREAD;

__device__ __forceinline__ int event_of(const int* hit_off, int n_events, int i) {
  int lo = 0, hi = n_events - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (hit_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_bin_count(const BinParams P) {
  const int i = P.h_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.h_end) return;
  const DevGeom& g = P.g;
  const int ev = event_of(P.hit_off, P.n_events, i);
  int l = P.hlayer[i];
  l = min(max(l, 0), g.n_layers - 1);
  const float x = P.hx[i], y = P.hy[i], z = P.hz[i];
  const int pb = wrap_bin(phi_bin_raw(atan2f(y, x), g.n_phi), g.n_phi);
  const int eb = eta_bin(z, g.radius[l], g.eta_max[l], g.n_eta, P.eta_edges + (size_t)l * (MAX_ETA_BINS + 1));
  const unsigned key =
      (unsigned)(((size_t)ev * g.n_layers + l) * ((size_t)g.n_eta * g.n_phi) + (size_t)eb * g.n_phi + pb);
  P.key[i] = key;
  P.rank[i] = atomicAdd(&P.cnt[key], 1u);
}

__global__ void k_bin_scatter(const BinParams P) {
  const int i = P.h_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.h_end) return;
  const int ev = event_of(P.hit_off, P.n_events, i);
  const unsigned pos = P.cnt[P.key[i]] + P.rank[i];
  P.hb[pos] = make_float4(P.hx[i], P.hy[i], P.hz[i], __int_as_float(i - P.hit_off[ev]));
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* sh, unsigned& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    unsigned w = lane < nw ? sh[lane] : 0u;
    unsigned wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < nw) sh[lane] = wi - w;
    if (lane == nw - 1) sh[32] = wi;
  }
  __syncthreads();
  total = sh[32];
  const unsigned r = sh[warp] + incl - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const unsigned* in, size_t n, unsigned* sums) {
  __shared__ unsigned sh[33];
  const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_PER_THREAD;
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k)
    if (base + k < n) s += in[base + k];
  unsigned total;
  block_exclusive_scan(s, sh, total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the tile sums in place; writes the grand
// total at sums[n_tiles].
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_sums(unsigned* sums, int n_tiles) {
  __shared__ unsigned sh[33];
  const int per = (n_tiles + SCAN_THREADS - 1) / SCAN_THREADS;
  const int b = threadIdx.x * per;
  unsigned s = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < n_tiles) s += sums[b + k];
  unsigned total;
  unsigned run = block_exclusive_scan(s, sh, total);
  for (int k = 0; k < per; ++k)
    if (b + k < n_tiles) {
      const unsigned v = sums[b + k];
      sums[b + k] = run;
      run += v;
    }
  if (threadIdx.x == 0) sums[n_tiles] = total;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(unsigned* data, size_t n, const unsigned* sums,
                                                             int n_tiles, unsigned add) {
  __shared__ unsigned sh[33];
  const size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_PER_THREAD;
  unsigned v[SCAN_PER_THREAD];
  unsigned s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    v[k] = (base + k < n) ? data[base + k] : 0u;
    s += v[k];
  }
  unsigned total;
  unsigned run = block_exclusive_scan(s, sh, total) + sums[blockIdx.x] + add;
#pragma unroll
  for (int k = 0; k < SCAN_PER_THREAD; ++k) {
    if (base + k < n) data[base + k] = run;
    run += v[k];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) data[n] = sums[n_tiles] + add;
}

}  // namespace

size_t scan_tmp_elems(size_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// Exclusive scan of cnt[0..n) in place plus `add`; cnt[n] = total + add.
static cudaError_t scan_inplace(unsigned* cnt, size_t n, unsigned add, unsigned* tmp, size_t tmp_elems,
                                cudaStream_t st) {
  const int n_tiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
  if ((size_t)n_tiles + 1 > tmp_elems) return cudaErrorInvalidValue;
  k_scan_reduce<<<n_tiles, SCAN_THREADS, 0, st>>>(cnt, n, tmp);
  k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(tmp, n_tiles);
  k_scan_apply<<<n_tiles, SCAN_THREADS, 0, st>>>(cnt, n, tmp, n_tiles, add);
  return cudaGetLastError();
}

// Bins the hits [P.h_begin, P.h_end), which must be whole events whose cells
// are cnt[bin_begin, bin_begin + n_bins); `first_pos` is the binned position
// of the first of them (the number of hits of all earlier events).
cudaError_t launch_bin(const BinParams& P, size_t bin_begin, size_t n_bins, unsigned first_pos,
                       unsigned* scan_tmp, size_t scan_tmp_elems_, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(P.cnt + bin_begin, 0, (n_bins + 1) * sizeof(unsigned), st);
  if (err != cudaSuccess) return err;
  const int n = P.h_end - P.h_begin;
  const int threads = 256;
  const int blocks = (n + threads - 1) / threads;
  if (n > 0) k_bin_count<<<blocks, threads, 0, st>>>(P);
  err = scan_inplace(P.cnt + bin_begin, n_bins, first_pos, scan_tmp, scan_tmp_elems_, st);
  if (err != cudaSuccess) return err;
  if (n > 0) k_bin_scatter<<<blocks, threads, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace kfg
