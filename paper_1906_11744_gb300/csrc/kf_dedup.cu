// Duplicate removal after building (the paper's post-processing step, Sec. 4.2).
//
// Definition (sequential): visit the tracks of an event by (more hits, lower
// chi2 sum, lower index); keep a track unless it shares more than
// frac * min(nA, nB) hits with a track already kept.
//
// Parallel form, identical result:
//   1. hit -> owning tracks table (count, exclusive scan, fill);
//   2. for every track, the shared-hit counts with every other track through
//      that table; a pair over the threshold is a conflict, recorded at the
//      lower-priority track;
//   3. resolution rounds: an undecided track is removed as soon as one of its
//      higher-priority conflicts is kept, and kept as soon as all of them are
//      removed.  The decisions equal the sequential walk's, because each one
//      only depends on the final decisions of higher-priority tracks; every
//      round settles at least the highest-priority undecided track.
// Batched launch: steps 1-2 one thread per track over the whole batch (the
// scan over every event's table at once), step 3 one block per event.
// Single-event launch (per-event form, allocation-free entry): all three
// steps in one block.
// Scratch (the owner table, the conflict lists and the decision states) lives
// in global memory owned by the caller.
#include <mutex>

#include "kf_internal.h"

namespace kfg {

namespace {

constexpr int DEDUP_THREADS = 1024;

__device__ __forceinline__ bool prio_less(int na, float ca, int ia, int nb, float cb, int ib) {
  if (na != nb) return na > nb;
  if (ca != cb) return ca < cb;
  return ia < ib;
}

// Owner-table count and fill of track t; cnt is its event's table.
__device__ __forceinline__ void dd_count(const DedupParams& P, int t, unsigned* cnt) {
  const int n = P.out_n[t];
  const int* ht = P.out_hits + (size_t)t * P.L;
  for (int j = 0; j < n; ++j) atomicAdd(&cnt[ht[j]], 1u);
}
__device__ __forceinline__ void dd_fill(const DedupParams& P, int t, unsigned* cnt, int* owners) {
  const int n = P.out_n[t];
  const int* ht = P.out_hits + (size_t)t * P.L;
  for (int j = 0; j < n; ++j) owners[atomicAdd(&cnt[ht[j]], 1u)] = t;
}

// Conflicts of track t (after the fill, hit h's owners are
// owners[start(h), cnt[h]) with start(h) = cnt[h - 1], start(0) = start0);
// resets its decision state.
__device__ __forceinline__ void dd_conflicts(const DedupParams& P, int t, const unsigned* cnt, unsigned start0,
                                             const int* owners) {
  const int n = P.out_n[t];
  const float c = P.out_chi2[t];
  const int* ht = P.out_hits + (size_t)t * P.L;
  int pid[DEDUP_PARTNER_CAP];
  int pcnt[DEDUP_PARTNER_CAP];
  int np = 0;
  bool overflow = false;
  for (int j = 0; j < n; ++j) {
    const int h = ht[j];
    const unsigned a = h == 0 ? start0 : cnt[h - 1], b = cnt[h];
    for (unsigned q = a; q < b; ++q) {
      const int u = owners[q];
      if (u == t) continue;
      int k = 0;
      while (k < np && pid[k] != u) ++k;
      if (k < np) {
        pcnt[k]++;
      } else if (np < DEDUP_PARTNER_CAP) {
        pid[np] = u;
        pcnt[np] = 1;
        ++np;
      } else {
        overflow = true;
      }
    }
  }
  if (overflow) atomicCAS(P.status, ST_OK, ST_DEDUP_PARTNERS);
  int nc = 0;
  for (int k = 0; k < np; ++k) {
    const int u = pid[k];
    const int nu = P.out_n[u];
    if ((float)pcnt[k] > P.frac * (float)min(n, nu) && prio_less(nu, P.out_chi2[u], u, n, c, t)) {
      if (nc < DEDUP_CONF_CAP) P.conf[(size_t)t * DEDUP_CONF_CAP + nc] = u;
      else atomicCAS(P.status, ST_OK, ST_DEDUP_CONFLICTS);
      ++nc;
    }
  }
  P.n_conf[t] = min(nc, DEDUP_CONF_CAP);
  P.state[t] = 0;  // undecided
}

// Resolution rounds of event e's tracks [s0, s1) by the whole block, then the
// keep flags.
__device__ void dd_rounds(const DedupParams& P, int s0, int s1) {
  __shared__ int sh_flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int max_rounds = (s1 - s0) + 2;  // bounded by the number of tracks
  int round = 0;
  for (;;) {
    if (tid == 0) sh_flag = 0;
    __syncthreads();
    int undecided = 0;
    for (int t = s0 + tid; t < s1; t += nt) {
      if (P.state[t] != 0) continue;
      const int nc = P.n_conf[t];
      bool any_kept = false, all_removed = true;
      for (int k = 0; k < nc; ++k) {
        const unsigned char s = ((volatile unsigned char*)P.state)[P.conf[(size_t)t * DEDUP_CONF_CAP + k]];
        if (s == 1) any_kept = true;
        if (s != 2) all_removed = false;
      }
      if (any_kept) P.state[t] = 2;
      else if (all_removed) P.state[t] = 1;
      else undecided = 1;
    }
    if (undecided) sh_flag = 1;
    __syncthreads();
    const int more = sh_flag;
    __syncthreads();
    if (!more) break;
    if (++round > max_rounds) {
      if (tid == 0) atomicCAS(P.status, ST_OK, ST_DEDUP_ROUNDS);
      break;
    }
  }
  for (int t = s0 + tid; t < s1; t += nt) P.keep[t] = P.state[t] == 1 ? 1 : 0;
}

__global__ void __launch_bounds__(DEDUP_THREADS) k_dedup(const DedupParams P) {
  __shared__ unsigned sh_scan[33];
  const int e = P.e_begin + blockIdx.x;
  const int s0 = P.seed_off[e], s1 = P.seed_off[e + 1];
  const int h0 = P.hit_off[e], h1 = P.hit_off[e + 1];
  const int nh = h1 - h0;
  const int L = P.L;
  unsigned* cnt = P.hit_cnt + h0 + e;   // nh + 1 entries per event
  int* owners = P.owners + (size_t)s0 * L;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int i = tid; i <= nh; i += nt) cnt[i] = 0u;
  __syncthreads();
  for (int t = s0 + tid; t < s1; t += nt) dd_count(P, t, cnt);
  __syncthreads();
  // block exclusive scan of cnt[0..nh)
  {
    const int per = (nh + nt - 1) / nt;
    const int b = tid * per;
    unsigned s = 0;
    for (int k = 0; k < per; ++k)
      if (b + k < nh) s += cnt[b + k];
    // inline block scan
    const int lane = tid & 31, warp = tid >> 5;
    unsigned incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) sh_scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const int nw = nt >> 5;
      unsigned w = lane < nw ? sh_scan[lane] : 0u, wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += v;
      }
      if (lane < nw) sh_scan[lane] = wi - w;
    }
    __syncthreads();
    unsigned run = sh_scan[warp] + incl - s;
    for (int k = 0; k < per; ++k)
      if (b + k < nh) {
        const unsigned v = cnt[b + k];
        cnt[b + k] = run;
        run += v;
      }
  }
  __syncthreads();
  // fill: afterwards cnt[h] is the end of hit h's owner range, cnt[h-1] its start
  for (int t = s0 + tid; t < s1; t += nt) dd_fill(P, t, cnt, owners);
  __syncthreads();
  for (int t = s0 + tid; t < s1; t += nt) dd_conflicts(P, t, cnt, 0u, owners);
  __syncthreads();
  dd_rounds(P, s0, s1);
}

// Batched steps, one thread per track of the whole batch.  Event e's table
// is hit_cnt[hit_off[e] + e, hit_off[e + 1] + e] (one extra entry); one
// exclusive scan over all tables makes the owner positions global.
__device__ __forceinline__ unsigned* dd_table(const DedupParams& P, int t, int& e) {
  e = P.seed_event[t];
  return P.hit_cnt + P.hit_off[e] + e;
}
__global__ void k_dd_count(const DedupParams P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.ns) return;
  int e;
  dd_count(P, t, dd_table(P, t, e));
}
__global__ void k_dd_fill(const DedupParams P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.ns) return;
  int e;
  dd_fill(P, t, dd_table(P, t, e), P.owners);
}
__global__ void k_dd_conflicts(const DedupParams P) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= P.ns) return;
  int e;
  const unsigned* cnt = dd_table(P, t, e);
  // hit 0's owners start where the previous table's extra entry points
  const unsigned start0 = (P.hit_off[e] + e == 0) ? 0u : cnt[-1];
  dd_conflicts(P, t, cnt, start0, P.owners);
}
__global__ void __launch_bounds__(DEDUP_THREADS) k_dd_rounds(const DedupParams P) {
  const int e = blockIdx.x;
  dd_rounds(P, P.seed_off[e], P.seed_off[e + 1]);
}

}  // namespace

cudaError_t launch_dedup(const DedupParams& P, int n_events, cudaStream_t st) {
  if (n_events <= 0) return cudaSuccess;
  k_dedup<<<n_events, DEDUP_THREADS, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_dedup_batched(const DedupParams& P, int n_events, int n_hits, unsigned* scan_tmp,
                                 size_t scan_tmp_elems_, cudaStream_t st) {
  if (n_events <= 0) return cudaSuccess;
  const size_t n_tab = (size_t)n_hits + n_events;
  cudaError_t e = cudaMemsetAsync(P.hit_cnt, 0, sizeof(unsigned) * (n_tab + 1), st);
  if (e != cudaSuccess) return e;
  const int threads = 256, blocks = (P.ns + threads - 1) / threads;
  if (P.ns > 0) k_dd_count<<<blocks, threads, 0, st>>>(P);
  e = scan_exclusive_inplace(P.hit_cnt, n_tab, 0u, scan_tmp, scan_tmp_elems_, st);
  if (e != cudaSuccess) return e;
  if (P.ns > 0) {
    k_dd_fill<<<blocks, threads, 0, st>>>(P);
    k_dd_conflicts<<<blocks, threads, 0, st>>>(P);
  }
  k_dd_rounds<<<n_events, DEDUP_THREADS, 0, st>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free duplicate removal (kf_remove_duplicates_noalloc).
//
// Some callers cannot allocate device memory at all: code that runs inside a
// host framework which owns every device allocation through its own pool, a
// trigger-style pipeline that forbids cudaMalloc/cudaFree on its hot path
// because they synchronize the device, or a plugin living within another
// library's fixed memory budget.  For them the duplicate-removal kernel also
// runs on a fixed scratch area in a file-scope device array, sized for one
// event of at most KF_NOALLOC_MAX_TRACKS tracks and KF_NOALLOC_MAX_HITS hits.
// The array exists once per device that loads the library and stays until the
// process exits.  Every call shares it: two calls whose kernels overlap on the
// GPU (different streams, or different host threads) race and give undefined
// results, so such calls must be ordered.
namespace {

constexpr size_t NA_CNT_BYTES = ((size_t)(KF_NOALLOC_MAX_HITS + 1) * 4 + 255) / 256 * 256;
constexpr size_t NA_OWN_BYTES = (size_t)KF_NOALLOC_MAX_TRACKS * KF_MAX_LAYERS * 4;
constexpr size_t NA_CONF_BYTES = (size_t)KF_NOALLOC_MAX_TRACKS * DEDUP_CONF_CAP * 4;
constexpr size_t NA_NCONF_BYTES = (size_t)KF_NOALLOC_MAX_TRACKS * 4;
constexpr size_t NA_STATE_BYTES = ((size_t)KF_NOALLOC_MAX_TRACKS + 255) / 256 * 256;
constexpr size_t NA_MISC_BYTES = 256;  // event offsets and the status word
constexpr size_t NA_BYTES =
    NA_CNT_BYTES + NA_OWN_BYTES + NA_CONF_BYTES + NA_NCONF_BYTES + NA_STATE_BYTES + NA_MISC_BYTES;

static __device__ __align__(256) unsigned char kf_noalloc_scratch[NA_BYTES];

// Device address of the scratch array per device, found once per device.
constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
unsigned char* na_ptr[NA_MAX_DEVICES] = {};

// Writes the one-event offsets and clears the status words.
__global__ void k_noalloc_prep(int* misc, int n_tracks, int n_hits, int* user_status) {
  if (threadIdx.x == 0) {
    misc[0] = 0;         // seed_off
    misc[1] = n_tracks;
    misc[2] = 0;         // hit_off
    misc[3] = n_hits;
    misc[4] = ST_OK;     // status
    if (user_status) *user_status = ST_OK;
  }
}

}  // namespace

}  // namespace kfg

extern "C" int kf_remove_duplicates_noalloc(int n_tracks, int n_layers, int n_hits, const int* hits,
                                            const int* n_found, const float* chi2, float dup_shared_frac,
                                            unsigned char* keep, int* status, void* stream) {
  using namespace kfg;
  if (n_tracks < 0 || n_hits < 0 || n_layers < 1 || n_layers > KF_MAX_LAYERS || !(dup_shared_frac >= 0.f))
    return KF_ERR_ARG;
  if (n_tracks > KF_NOALLOC_MAX_TRACKS || n_hits > KF_NOALLOC_MAX_HITS) return KF_ERR_CAPACITY;
  if (n_tracks == 0) return KF_OK;
  if (!hits || !n_found || !chi2 || !keep) return KF_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return KF_ERR_CUDA;
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, kf_noalloc_scratch) != cudaSuccess || !p) return KF_ERR_CUDA;
      na_ptr[dev] = static_cast<unsigned char*>(p);
    }
    base = na_ptr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int* misc = reinterpret_cast<int*>(base + NA_BYTES - NA_MISC_BYTES);
  DedupParams D;
  D.out_hits = hits;
  D.out_n = n_found;
  D.out_chi2 = chi2;
  D.seed_off = misc;
  D.seed_event = nullptr;  // single-event launch only
  D.hit_off = misc + 2;
  D.L = n_layers;
  D.ns = n_tracks;
  D.frac = dup_shared_frac;
  D.e_begin = 0;
  D.hit_cnt = reinterpret_cast<unsigned*>(base);
  D.owners = reinterpret_cast<int*>(base + NA_CNT_BYTES);
  D.conf = reinterpret_cast<int*>(base + NA_CNT_BYTES + NA_OWN_BYTES);
  D.n_conf = reinterpret_cast<int*>(base + NA_CNT_BYTES + NA_OWN_BYTES + NA_CONF_BYTES);
  D.state = base + NA_CNT_BYTES + NA_OWN_BYTES + NA_CONF_BYTES + NA_NCONF_BYTES;
  D.keep = keep;
  D.status = status ? status : misc + 4;
  k_noalloc_prep<<<1, 32, 0, st>>>(misc, n_tracks, n_hits, status);
  if (cudaGetLastError() != cudaSuccess) return KF_ERR_CUDA;
  if (launch_dedup(D, 1, st) != cudaSuccess) return KF_ERR_CUDA;
  return KF_OK;
}
