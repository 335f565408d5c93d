// Duplicate handling (Sec. 4.2): seed cleaning before building and duplicate
// removal after it.
//
// Kinematic closeness of two tracks or seeds (the paper names pT, eta and phi
// as criteria of both steps): |d eta| < deta, |d phi0| < dphi (difference on
// the circle), ||k_A| - |k_B|| <= dpt max(|k_A|, |k_B|) with k = q/pT; a cut
// <= 0 is not applied.  eta = -ln tan(theta/2); phi0 is the direction of
// motion at the point of the helix closest to the z axis, which every state
// along the helix shares.
//
// Duplicate removal, definition (sequential): visit the tracks of an event by
// (more hits, lower chi2 sum, lower index); keep a track unless it shares more
// than frac * min(nA, nB) hits with a track already kept and (with the
// kinematic pre-cuts) is kinematically close to it.  A track without hits (a
// cleaned seed's) is never kept.
//
// Seed cleaning, definition (sequential): visit the seeds of an event by
// index; drop a seed when a seed already kept is kinematically close to it and
// shares at least min_shared of its three hits.  Parallel form: the same
// conflict lists and resolution rounds as below, the pairs found by scanning
// each seed's neighbours in the theta order of the event.
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

// (eta, phi0, |q/pT|) of a state.  phi0 = atan2(-v_x, v_y) with
// v = h c = (h x - sin phi, h y + cos phi), h times the centre c of the track
// circle: the closest point to the axis lies along c, where the direction of
// motion is sign(h) (c_y, -c_x)/|c|.  For h = 0, v = (-sin phi, cos phi) and
// phi0 = phi.  Accurate library functions: these values decide which tracks
// are kept.
struct Kin {
  float eta, phi0, ak;
};
__device__ __forceinline__ Kin kin_of(float x, float y, float kappa, float phi, float theta, float kb) {
  const float h = kb * kappa;
  float s, c;
  sincosf(phi, &s, &c);
  Kin k;
  k.eta = -logf(tanf(0.5f * theta));
  k.phi0 = atan2f(-fmaf(h, x, -s), fmaf(h, y, c));
  k.ak = fabsf(kappa);
  return k;
}
__device__ __forceinline__ bool kin_close(const Kin& a, const Kin& b, float deta, float dphi, float dpt) {
  if (deta > 0.f && !(fabsf(a.eta - b.eta) < deta)) return false;
  if (dphi > 0.f) {
    float d = fabsf(a.phi0 - b.phi0);
    if (d > PI_F) d = TWO_PI_F - d;
    if (!(d < dphi)) return false;
  }
  if (dpt > 0.f && !(fabsf(a.ak - b.ak) <= dpt * fmaxf(a.ak, b.ak))) return false;
  return true;
}
// Kinematics of track t from its state [6][ns].
__device__ __forceinline__ Kin track_kin(const DedupParams& P, int t) {
  const float* q = P.trk_p + t;
  const size_t n = (size_t)P.ns;
  return kin_of(q[0], q[n], q[3 * n], q[4 * n], q[5 * n], P.kb);
}

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
  if (n == 0) {  // no track (a cleaned seed): removed, nothing to compare
    P.n_conf[t] = 0;
    P.state[t] = 2;
    return;
  }
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
  const bool kin = P.trk_p != nullptr;
  Kin kt;
  if (kin) kt = track_kin(P, t);
  int nc = 0;
  for (int k = 0; k < np; ++k) {
    const int u = pid[k];
    const int nu = P.out_n[u];
    if ((float)pcnt[k] > P.frac * (float)min(n, nu) && prio_less(nu, P.out_chi2[u], u, n, c, t) &&
        (!kin || kin_close(kt, track_kin(P, u), P.deta, P.dphi, P.dpt))) {
      if (nc < DEDUP_CONF_CAP) P.conf[(size_t)t * DEDUP_CONF_CAP + nc] = u;
      else atomicCAS(P.status, ST_OK, ST_DEDUP_CONFLICTS);
      ++nc;
    }
  }
  P.n_conf[t] = min(nc, DEDUP_CONF_CAP);
  P.state[t] = 0;  // undecided
}

// Resolution rounds of items [s0, s1) (an event's tracks or seeds) by the
// whole block, then the keep flags.  Each item's conflicts are the
// higher-priority items that remove it if kept.
struct Rounds {
  const int* n_conf;
  const int* conf;
  unsigned char* state;
  unsigned char* keep;
  int* status;
  int err;         // status value when the rounds do not settle
  int max_rounds;  // rounds before giving up; 0: n + 4, which always settles
};
// One step of item t: removed as soon as one of its conflicts is kept, kept
// as soon as all of them are removed.  Returns false while undecided.
__device__ __forceinline__ bool dd_decide(const Rounds& P, int t) {
  if (P.state[t] != 0) return true;
  const int nc = min(P.n_conf[t], DEDUP_CONF_CAP);
  bool any_kept = false, all_removed = true;
  for (int k = 0; k < nc; ++k) {
    const unsigned char s = ((volatile unsigned char*)P.state)[P.conf[(size_t)t * DEDUP_CONF_CAP + k]];
    if (s == 1) any_kept = true;
    if (s != 2) all_removed = false;
  }
  if (any_kept) P.state[t] = 2;
  else if (all_removed) P.state[t] = 1;
  else return false;
  return true;
}
// Rounds by the whole block over items item(0..n) until every one is decided
// (at most n + 2 rounds: each settles the highest-priority undecided item),
// or, with a round cap, until the cap (the status then records the failure).
template <class Item>
__device__ void dd_rounds_over(const Rounds& P, int n, Item item) {
  __shared__ int sh_flag;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int round = 0;; ++round) {
    if (tid == 0) sh_flag = 0;
    __syncthreads();
    bool undecided = false;
    for (int i = tid; i < n; i += nt)
      if (!dd_decide(P, item(i))) undecided = true;
    if (undecided) sh_flag = 1;
    __syncthreads();
    const int more = sh_flag;
    __syncthreads();
    if (!more) break;
    if (round + 1 >= (P.max_rounds > 0 ? P.max_rounds : n + 4)) {
      if (tid == 0) atomicCAS(P.status, ST_OK, P.err);
      break;
    }
  }
}
__device__ void dd_rounds(const Rounds& P, int s0, int s1) {
  dd_rounds_over(P, s1 - s0, [&](int i) { return s0 + i; });
  if (P.keep)
    for (int t = s0 + threadIdx.x; t < s1; t += blockDim.x) P.keep[t] = P.state[t] == 1 ? 1 : 0;
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
  dd_rounds(Rounds{P.n_conf, P.conf, P.state, P.keep, P.status, ST_DEDUP_ROUNDS, P.max_rounds}, s0, s1);
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
  dd_rounds(Rounds{P.n_conf, P.conf, P.state, P.keep, P.status, ST_DEDUP_ROUNDS, P.max_rounds}, P.seed_off[e],
            P.seed_off[e + 1]);
}

// ------------------------------------------------------------ seed cleaning
// Kinematics and hits of the seed at each position of the theta order; its
// conflict count cleared and its state preset to kept (a seed without
// conflicts is kept); the event's list of seeds with conflicts emptied.
__global__ void k_sc_kin(const SeedCleanParams P, int pos_begin, int pos_end) {
  const int j = pos_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= pos_end) return;
  const int e = P.seed_event[j];
  if (j == P.seed_off[e]) P.list_cnt[e] = 0;
  const int s = P.order[j];
  const size_t n = (size_t)P.ns;
  const float th = P.sp[5 * n + s];
  const Kin k = kin_of(P.sp[s], P.sp[n + s], P.sp[3 * n + s], P.sp[4 * n + s], th, P.kb);
  P.kin[j] = make_float4(k.eta, k.phi0, k.ak, __int_as_float(seed_theta_bin(th)));
  P.kseed[j] = make_int4(s, P.sh[s], P.sh[n + s], P.sh[2 * n + s]);
  P.n_conf[j] = 0;
  P.state[j] = 1;
}

// Duplicate pairs, each tested once: the seed at position j against the
// later positions of its event within its theta-bin window.  A pair found is
// a conflict of its higher-index seed (conflict lists and decision states are
// kept by position, so that the resolution reads them in order); a seed's
// first conflict makes it undecided and enters it in its event's list (at
// most one entry per position of the event).  The theta
// order is sorted by theta bin, and every seed within deta in eta of seed j
// has theta below theta(eta_j - deta), theta(eta) = 2 atan(exp(-eta)): the
// scan stops past that bin (one bin more absorbs rounding).  A later position
// in the same or a later bin can also lie below eta_j; both halves of the
// window are covered because the lower member of every pair scans upward.
__global__ void k_sc_conflicts(const SeedCleanParams P, int pos_begin, int pos_end) {
  const int j = pos_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= pos_end) return;
  const int e = P.seed_event[j];  // positions and seed indices share the event ranges
  const int lo = P.seed_off[e], hi = P.seed_off[e + 1];
  const float4 a4 = P.kin[j];
  const Kin a{a4.x, a4.y, a4.z};
  const int b_hi = seed_theta_bin(2.f * atanf(expf(-(a.eta - P.deta)))) + 1;
  int4 me = make_int4(-1, 0, 0, 0);
  for (int q = j + 1; q < hi; ++q) {
    const float4 b4 = P.kin[q];
    if (__float_as_int(b4.w) > b_hi) break;
    if (!kin_close(a, Kin{b4.x, b4.y, b4.z}, P.deta, P.dphi, P.dpt)) continue;
    if (me.x < 0) me = P.kseed[j];
    const int4 o = P.kseed[q];
    const int shared = (me.y == o.y) + (me.y == o.z) + (me.y == o.w) + (me.z == o.y) + (me.z == o.z) +
                       (me.z == o.w) + (me.w == o.y) + (me.w == o.z) + (me.w == o.w);
    if (shared < P.min_shared) continue;
    const int t = o.x > me.x ? q : j, u = o.x > me.x ? j : q;  // t is removed by u if u is kept
    const int slot = atomicAdd(&P.n_conf[t], 1);
    if (slot < DEDUP_CONF_CAP) P.conf[(size_t)t * DEDUP_CONF_CAP + slot] = u;
    else atomicCAS(P.status, ST_OK, ST_SEED_CONFLICTS);
    if (slot == 0) {
      P.state[t] = 0;
      P.list[lo + atomicAdd(&P.list_cnt[e], 1)] = t;
    }
  }
}

// Per event (one block): the resolution rounds over the event's seeds with
// conflicts; then the new order of its positions (kept seeds first in theta
// order, the dropped ones from the end) and the empty outputs of the dropped
// seeds.  Each thread splits a contiguous segment of positions; one block
// scan of the segments' kept counts places them.
__global__ void __launch_bounds__(DEDUP_THREADS) k_sc_resolve(const SeedCleanParams P, int e_begin) {
  __shared__ int s_warp[DEDUP_THREADS / 32];
  __shared__ int s_tot;
  const int e = e_begin + blockIdx.x;
  const int s0 = P.seed_off[e], s1 = P.seed_off[e + 1];
  if (s1 <= s0) {
    if (threadIdx.x == 0) P.kept_cnt[e] = 0;
    return;
  }
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int* list = P.list + s0;
  dd_rounds_over(Rounds{P.n_conf, P.conf, P.state, nullptr, P.status, ST_SEED_ROUNDS, P.max_rounds}, P.list_cnt[e],
                 [&](int i) { return list[i]; });
  __syncthreads();
  const int per = (s1 - s0 + nt - 1) / nt;
  const int a = min(s0 + tid * per, s1), b = min(a + per, s1);
  int mine = 0;
  for (int j = a; j < b; ++j) mine += P.state[j] == 1;
  // exclusive scan of the kept counts over the block
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < nw ? s_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    if (lane < nw) s_warp[lane] = wi - w;
    if (lane == nw - 1) s_tot = wi;
  }
  __syncthreads();
  int kr = s_warp[warp] + incl - mine;   // kept positions before this segment
  int dr = (a - s0) - kr;                // dropped positions before it
  const size_t n = (size_t)P.ns;
  for (int j = a; j < b; ++j) {
    const int s = P.order[j];
    if (P.state[j] == 1) {
      P.clean_order[s0 + kr++] = s;
    } else {
      P.clean_order[s1 - 1 - dr++] = s;
      P.keep[s] = 0;
      P.out_n[s] = 0;
      P.out_chi2[s] = 0.f;
      for (int l = 0; l < P.L; ++l) P.out_hits[(size_t)s * P.L + l] = -1;
      for (int k = 0; k < 6; ++k) P.out_p[k * n + s] = P.sp[k * n + s];
      for (int k = 0; k < 21; ++k) P.out_C[k * n + s] = P.sc[k * n + s];
    }
  }
  if (tid == 0) P.kept_cnt[e] = s_tot;
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

cudaError_t launch_seed_clean(const SeedCleanParams& P, int pos_begin, int pos_end, int e_begin, int n_events,
                              cudaStream_t st) {
  if (n_events <= 0) return cudaSuccess;
  const int n = pos_end - pos_begin;
  if (n > 0) {
    const int threads = 256, blocks = (n + threads - 1) / threads;
    k_sc_kin<<<blocks, threads, 0, st>>>(P, pos_begin, pos_end);
    k_sc_conflicts<<<blocks, threads, 0, st>>>(P, pos_begin, pos_end);
  }
  k_sc_resolve<<<n_events, DEDUP_THREADS, 0, st>>>(P, e_begin);
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
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (n_tracks == 0) {  // nothing to remove; the status still reads "no error"
    if (status && cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return KF_ERR_CUDA;
    return KF_OK;
  }
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
