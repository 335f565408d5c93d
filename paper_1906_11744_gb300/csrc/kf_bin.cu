// Hit binning: counting sort of every hit into its (event, surface, row, phi
// bin) cell, so that a search window is a few contiguous ranges of the
// binned array (the GPU form of the paper's per-layer hit search windows,
// Sec. 3).  On a barrel layer the grid is n_eta rows in eta = asinh(z/R_layer)
// over [-asinh(z_max/R), +asinh(z_max/R)] (as z edges per layer), on an
// endcap disk n_eta rows in r over [disk_rmin, disk_rmax]; times n_phi bins
// in phi = atan2(y, x).
//
// Layer-grouped form (grids of at most 65,536 cells per layer):
//   1. k_group_count / k_group_scan / k_group_scatter: counting sort of the
//      hits by (event, layer) (warp-aggregated atomics on E x L counters);
//   2. k_cells: one block per (event, layer) counts its hits per cell in
//      shared memory (two 16-bit counters per word, padded against bank
//      conflicts), scans the counts in place, writes the cell offsets
//      (coalesced) and scatters its hits.  A layer of one event with more
//      than 65,535 hits is done by its block with global counters instead.
// General form (larger grids): k_bin_count (key and rank of each hit by an
// atomic count per cell), an exclusive scan of the counts (three passes),
// k_bin_scatter (hit -> offset[key] + rank).
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

// Row of a hit in the grid of its surface l: the eta bin on a layer, the r
// bin on a disk.
__device__ __forceinline__ int row_of(const BinParams& P, int l, float x, float y, float z) {
  const DevGeom& g = P.g;
  if (is_disk(g, l)) return r_bin(g, disk_r(x, y));
  return eta_bin(z, g.n_eta, g.z_max, g.eta_lut_scale, P.eta_lut + (size_t)l * ETA_LUT,
                 P.eta_edges + (size_t)l * (MAX_ETA_BINS + 1));
}

// Cell of a hit within its surface's grid.
__device__ __forceinline__ int cell_of(const BinParams& P, int l, float x, float y, float z) {
  const DevGeom& g = P.g;
  const int pb = wrap_bin(phi_bin_raw(atan2f(y, x), g.phi_scale), g.n_phi);
  return row_of(P, l, x, y, z) * g.n_phi + pb;
}

__global__ void k_bin_count(const BinParams P) {
  const int i = P.h_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.h_end) return;
  const DevGeom& g = P.g;
  const int ev = event_of(P.hit_off, P.n_events, i);
  int l = P.hlayer[i];
  l = min(max(l, 0), g.n_surf - 1);
  const unsigned key = (unsigned)(((size_t)ev * g.n_surf + l) * ((size_t)g.n_eta * g.n_phi) +
                                  cell_of(P, l, P.hx[i], P.hy[i], P.hz[i]));
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

// ---- grouped form
// Buckets: (event, layer, chunk of eta rows) with at most CHUNK_CELLS cells.
constexpr int CHUNK_CELLS = 16384;
constexpr int CELL_THREADS = 256;
constexpr int CELL_WORDS = CHUNK_CELLS / 2;                    // two 16-bit counters per word
constexpr int CELL_SMEM_WORDS = CELL_WORDS + CELL_WORDS / 32;  // one pad word per 32
constexpr int GROUP_THREADS = 256;
constexpr int GROUP_HITS = 4096;  // hits of one event per grouping block
__device__ __forceinline__ int pad_word(int w) { return w + (w >> 5); }

struct Chunks {
  int rows;  // eta rows per chunk
  int n;     // chunks per layer
};
__host__ __device__ inline Chunks chunks_of(int n_eta, int n_phi) {
  Chunks c;
  c.rows = CHUNK_CELLS / n_phi < 1 ? 1 : CHUNK_CELLS / n_phi;
  if (c.rows > n_eta) c.rows = n_eta;
  c.n = (n_eta + c.rows - 1) / c.rows;
  return c;
}

// Bucket of hit i of event ev within the event (surface, chunk).
__device__ __forceinline__ int bucket_in_event(const BinParams& P, int i, Chunks ch) {
  const int l = min(max(P.hlayer[i], 0), P.g.n_surf - 1);
  return l * ch.n + row_of(P, l, P.hx[i], P.hy[i], P.hz[i]) / ch.rows;
}

// Grid (ceil(max event hits / GROUP_HITS), events of the launch): block (c, e)
// takes hits [GROUP_HITS c, GROUP_HITS (c + 1)) of event e_first + e.
// COUNT: per-block histogram of the event's buckets added to the global
// counts.  SCATTER: per-block bases from the global cursors, hits written to
// the grouped array at base + rank within the block.
template <bool COUNT>
__global__ void __launch_bounds__(GROUP_THREADS) k_group(const BinParams P, int e_first, int n_buckets) {
  extern __shared__ unsigned hist[];  // buckets of one event
  const Chunks ch = chunks_of(P.g.n_eta, P.g.n_phi);
  const int nb_ev = P.g.n_surf * ch.n;
  const int ev = e_first + blockIdx.y;
  const int h0 = P.hit_off[ev] + blockIdx.x * GROUP_HITS;
  const int h1 = min(P.hit_off[ev + 1], h0 + GROUP_HITS);
  if (h0 >= h1) return;
  for (int k = threadIdx.x; k < nb_ev; k += blockDim.x) hist[k] = 0u;
  __syncthreads();
  unsigned* gcnt = P.gtab + (size_t)blockIdx.y * nb_ev;
  if (COUNT) {
    for (int i = h0 + threadIdx.x; i < h1; i += blockDim.x) atomicAdd(&hist[bucket_in_event(P, i, ch)], 1u);
    __syncthreads();
    for (int k = threadIdx.x; k < nb_ev; k += blockDim.x)
      if (hist[k]) atomicAdd(&gcnt[k], hist[k]);
  } else {
    unsigned* bases = hist + nb_ev;
    for (int i = h0 + threadIdx.x; i < h1; i += blockDim.x) atomicAdd(&hist[bucket_in_event(P, i, ch)], 1u);
    __syncthreads();
    unsigned* gcur = P.gtab + 2 * (size_t)n_buckets + 2 + (size_t)blockIdx.y * nb_ev;
    const unsigned first = P.gtab[n_buckets + 1];
    for (int k = threadIdx.x; k < nb_ev; k += blockDim.x) {
      bases[k] = hist[k] ? atomicAdd(&gcur[k], hist[k]) - first : 0u;
      hist[k] = 0u;
    }
    __syncthreads();
    for (int i = h0 + threadIdx.x; i < h1; i += blockDim.x) {
      const int bk = bucket_in_event(P, i, ch);
      const unsigned pos = bases[bk] + atomicAdd(&hist[bk], 1u);
      P.grouped[pos] = make_float4(P.hx[i], P.hy[i], P.hz[i], __int_as_float(i - P.hit_off[ev]));
    }
  }
}

// One block: exclusive scan of the n bucket counts (plus first_pos) into
// gtab[n + 1 ..] (bases, with the total after the last) and gtab[2n + 2 ..]
// (cursors); the total also closes the cell offsets at cnt[end_cell].
__global__ void __launch_bounds__(SCAN_THREADS) k_group_scan(const BinParams P, int n, unsigned first_pos,
                                                             size_t end_cell) {
  __shared__ unsigned sh[33];
  const int per = (n + SCAN_THREADS - 1) / SCAN_THREADS;
  const int b = threadIdx.x * per;
  unsigned s = 0;
  for (int k = 0; k < per; ++k)
    if (b + k < n) s += P.gtab[b + k];
  unsigned total;
  unsigned run = block_exclusive_scan(s, sh, total) + first_pos;
  for (int k = 0; k < per; ++k)
    if (b + k < n) {
      P.gtab[n + 1 + b + k] = run;
      P.gtab[2 * n + 2 + b + k] = run;
      run += P.gtab[b + k];
    }
  if (threadIdx.x == 0) {
    P.gtab[n + 1 + n] = total + first_pos;
    P.cnt[end_cell] = total + first_pos;
  }
}

// One block per bucket (event, layer, chunk of eta rows) of the launch:
// counts per cell in shared memory, exclusive scan in place, cell offsets
// written (coalesced), hits scattered.  A bucket above 65,535 hits takes
// global counters instead (the general form's steps, within this block).
__global__ void __launch_bounds__(CELL_THREADS) k_cells(const BinParams P, int e_first, int n_buckets) {
  extern __shared__ unsigned cw[];  // CELL_SMEM_WORDS
  __shared__ unsigned sh[33];
  const Chunks ch = chunks_of(P.g.n_eta, P.g.n_phi);
  const int b = blockIdx.x;
  const int chunk = b % ch.n;
  const int l = (b / ch.n) % P.g.n_surf;
  const int ev_rel = b / (ch.n * P.g.n_surf);
  const int n_phi = P.g.n_phi;
  const int row0 = chunk * ch.rows;
  const int C = min(ch.rows, P.g.n_eta - row0) * n_phi;  // cells of the chunk
  const unsigned first = P.gtab[n_buckets + 1];
  const unsigned g0 = P.gtab[n_buckets + 1 + b], g1 = P.gtab[n_buckets + 2 + b];
  const int n = (int)(g1 - g0);
  const float4* hits = P.grouped + (g0 - first);
  unsigned* off = P.cnt + ((size_t)(e_first + ev_rel) * P.g.n_surf + l) * ((size_t)P.g.n_eta * n_phi) +
                  (size_t)row0 * n_phi;
  const int tid = threadIdx.x;
  auto cell = [&](const float4& h) {
    return (row_of(P, l, h.x, h.y, h.z) - row0) * n_phi + wrap_bin(phi_bin_raw(atan2f(h.y, h.x), P.g.phi_scale), n_phi);
  };
  if (n > 65535) {
    for (int c = tid; c < C; c += CELL_THREADS) off[c] = 0u;
    __syncthreads();
    for (int k = tid; k < n; k += CELL_THREADS) {
      const int c = cell(hits[k]);
      P.key[g0 - first + k] = (unsigned)c;
      P.rank[g0 - first + k] = atomicAdd(&off[c], 1u);
    }
    __syncthreads();
    const int per = (C + CELL_THREADS - 1) / CELL_THREADS;
    unsigned s = 0;
    for (int k = 0; k < per; ++k)
      if (tid * per + k < C) s += off[tid * per + k];
    unsigned total;
    unsigned run = block_exclusive_scan(s, sh, total) + g0;
    for (int k = 0; k < per; ++k)
      if (tid * per + k < C) {
        const unsigned v = off[tid * per + k];
        off[tid * per + k] = run;
        run += v;
      }
    __syncthreads();
    for (int k = tid; k < n; k += CELL_THREADS) P.hb[off[P.key[g0 - first + k]] + P.rank[g0 - first + k]] = hits[k];
    return;
  }
  for (int w = tid; w < CELL_SMEM_WORDS; w += CELL_THREADS) cw[w] = 0u;
  __syncthreads();
  for (int k = tid; k < n; k += CELL_THREADS) {
    const int c = cell(hits[k]);
    atomicAdd(&cw[pad_word(c >> 1)], 1u << ((c & 1) * 16));
  }
  __syncthreads();
  // exclusive scan in place: thread t owns words [32t, 32t + 32) (64 cells)
  {
    unsigned* my = cw + pad_word(tid * 32);  // 32 consecutive padded words
    unsigned s = 0;
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const unsigned w = my[k];
      s += (w & 0xFFFFu) + (w >> 16);
    }
    unsigned total;
    unsigned run = block_exclusive_scan(s, sh, total);
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const unsigned w = my[k];
      const unsigned lo = run;
      const unsigned hi = run + (w & 0xFFFFu);
      run = hi + (w >> 16);
      my[k] = lo | (hi << 16);
    }
  }
  __syncthreads();
  for (int c = tid; c < C; c += CELL_THREADS) {
    const unsigned w = cw[pad_word(c >> 1)];
    off[c] = g0 + ((c & 1) ? (w >> 16) : (w & 0xFFFFu));
  }
  __syncthreads();
  for (int k = tid; k < n; k += CELL_THREADS) {
    const float4 h = hits[k];
    const int c = cell(h);
    const unsigned old = atomicAdd(&cw[pad_word(c >> 1)], 1u << ((c & 1) * 16));
    P.hb[g0 + ((c & 1) ? (old >> 16) : (old & 0xFFFFu))] = h;
  }
}

}  // namespace

size_t scan_tmp_elems(size_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

// Exclusive scan of cnt[0..n) in place plus `add`; cnt[n] = total + add.
cudaError_t scan_exclusive_inplace(unsigned* cnt, size_t n, unsigned add, unsigned* tmp, size_t tmp_elems,
                                   cudaStream_t st) {
  const int n_tiles = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
  if ((size_t)n_tiles + 1 > tmp_elems) return cudaErrorInvalidValue;
  k_scan_reduce<<<n_tiles, SCAN_THREADS, 0, st>>>(cnt, n, tmp);
  k_scan_sums<<<1, SCAN_THREADS, 0, st>>>(tmp, n_tiles);
  k_scan_apply<<<n_tiles, SCAN_THREADS, 0, st>>>(cnt, n, tmp, n_tiles, add);
  return cudaGetLastError();
}

size_t bin_group_elems(int n_events, int n_layers, int n_eta, int n_phi) {
  return 3 * ((size_t)n_events * n_layers * chunks_of(n_eta, n_phi).n + 1);
}

// Bins the hits [P.h_begin, P.h_end), which must be whole events whose cells
// are cnt[bin_begin, bin_begin + n_bins); `first_pos` is the binned position
// of the first of them (the number of hits of all earlier events).
// max_event_hits: the largest hit count of those events.
cudaError_t launch_bin(const BinParams& P, size_t bin_begin, size_t n_bins, unsigned first_pos, int max_event_hits,
                       unsigned* scan_tmp, size_t scan_tmp_elems_, cudaStream_t st) {
  const int n_hits = P.h_end - P.h_begin;
  if (P.g.n_phi <= CHUNK_CELLS && P.grouped && P.gtab) {
    const Chunks ch = chunks_of(P.g.n_eta, P.g.n_phi);
    const size_t per_event = (size_t)P.g.n_surf * P.g.n_eta * P.g.n_phi;
    const int e_first = (int)(bin_begin / per_event);
    const int n_ev = (int)(n_bins / per_event);
    const int nb_ev = P.g.n_surf * ch.n;
    const int nb = n_ev * nb_ev;  // buckets of the launch
    cudaError_t err = cudaMemsetAsync(P.gtab, 0, sizeof(unsigned) * (size_t)nb, st);
    if (err != cudaSuccess) return err;
    const dim3 ggrid((max_event_hits + GROUP_HITS - 1) / GROUP_HITS, n_ev);
    if (n_hits > 0 && ggrid.x > 0) k_group<true><<<ggrid, GROUP_THREADS, sizeof(unsigned) * nb_ev, st>>>(P, e_first, nb);
    k_group_scan<<<1, SCAN_THREADS, 0, st>>>(P, nb, first_pos, bin_begin + n_bins);
    if (n_hits > 0 && ggrid.x > 0)
      k_group<false><<<ggrid, GROUP_THREADS, 2 * sizeof(unsigned) * nb_ev, st>>>(P, e_first, nb);
    const size_t smem = sizeof(unsigned) * CELL_SMEM_WORDS;
    if (nb > 0) k_cells<<<nb, CELL_THREADS, smem, st>>>(P, e_first, nb);
    return cudaGetLastError();
  }
  cudaError_t err = cudaMemsetAsync(P.cnt + bin_begin, 0, (n_bins + 1) * sizeof(unsigned), st);
  if (err != cudaSuccess) return err;
  const int threads = 256;
  const int blocks = (n_hits + threads - 1) / threads;
  if (n_hits > 0) k_bin_count<<<blocks, threads, 0, st>>>(P);
  err = scan_exclusive_inplace(P.cnt + bin_begin, n_bins, first_pos, scan_tmp, scan_tmp_elems_, st);
  if (err != cudaSuccess) return err;
  if (n_hits > 0) k_bin_scatter<<<blocks, threads, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace kfg
