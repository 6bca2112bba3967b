// sg_sim.cu -- kernels and C entry points of the vectorized Sparrow simulator
// (paper arxiv 2305.04180, Sec. 3.2).  See include/sparrow_gb.h for the
// contract of every extern "C" function.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sg_device.cuh"
#include "sg_host.h"
#include "sparrow_gb.h"

using namespace sg;

// ------------------------------------------------------------------ kernels

// ---------------------------------------------------------------- maps
// Map preprocessing runs over a group of maps staged together on the device:
// item counts (words, rows, cells) are prefix-summed per map, and every
// thread finds its map by binary search over the prefix.
struct PrepMap {
  long long src;        // first cell of the map in the staging grid
  long long word_off;   // first word in the bit atlas
  long long clr_off;    // interior cell (0, 0) in the skip-map atlas
  int w, h, row_words, clr_ld;
};

__device__ __forceinline__ int find_map(const long long* __restrict__ prefix, int n_maps, long long item) {
  int lo = 0, hi = n_maps - 1;  // largest m with prefix[m] <= item
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Bits: warp per (map, row word); bit b of the word is cell 32 * word + b (a ballot).
__global__ void k_pack_maps(const uint8_t* __restrict__ grid, const PrepMap* __restrict__ mp,
                            const long long* __restrict__ word_prefix, int n_maps, long long total,
                            uint32_t* __restrict__ atlas) {
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= total) return;  // warp-uniform
  const int m = find_map(word_prefix, n_maps, gw);
  const PrepMap d = mp[m];
  const long long local = gw - word_prefix[m];
  const int cy = (int)(local / d.row_words), wd = (int)(local % d.row_words);
  const int cx = wd * 32 + lane;
  const bool occ = cx < d.w && grid[d.src + (long long)cy * d.w + cx] != 0;
  const uint32_t word = __ballot_sync(kFull, occ);
  if (lane == 0) atlas[d.word_off + local] = word;
}

// Clearance, pass 1: thread per (map, row): distance along the row to the
// nearest occupied cell (outside counts as occupied), capped at 255.
__global__ void k_clr_rows(const uint8_t* __restrict__ grid, const PrepMap* __restrict__ mp,
                           const long long* __restrict__ row_prefix, int n_maps, long long total,
                           uint8_t* __restrict__ g) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= total) return;
  const int m = find_map(row_prefix, n_maps, r);
  const PrepMap d = mp[m];
  const int cy = (int)(r - row_prefix[m]);
  const uint8_t* row = grid + d.src + (long long)cy * d.w;
  uint8_t* out = g + d.src + (long long)cy * d.w;
  int dist = 0;  // to the last occupied cell on the left (x = -1 is outside)
  for (int cx = 0; cx < d.w; ++cx) {
    dist = row[cx] ? 0 : dist + 1;
    out[cx] = (uint8_t)min(dist, 255);
  }
  dist = 0;
  for (int cx = d.w - 1; cx >= 0; --cx) {
    dist = row[cx] ? 0 : dist + 1;
    out[cx] = (uint8_t)min((int)out[cx], min(dist, 255));
  }
}

// Pass 2: thread per (map, cell): Chebyshev distance
// d(x, y) = min over rows y' of max(g(x, y'), |y - y'|), with the rows outside
// the map at g = 0; capped at 255; stored as the march's skip value
// (0 if d = 0, else max(1, d - 1)) inside the zero border.
__global__ void k_clr_cols(const uint8_t* __restrict__ g, const PrepMap* __restrict__ mp,
                           const long long* __restrict__ cell_prefix, int n_maps, long long total,
                           uint8_t* __restrict__ clr) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int m = find_map(cell_prefix, n_maps, i);
  const PrepMap d = mp[m];
  const long long local = i - cell_prefix[m];
  const int cx = (int)(local % d.w), cy = (int)(local / d.w);
  const uint8_t* col = g + d.src + cx;
  int best = min(min(cy + 1, d.h - cy), 255);
  for (int dd = 0; dd < best; ++dd) {
    if (cy - dd >= 0) best = min(best, max((int)col[(long long)(cy - dd) * d.w], dd));
    if (cy + dd < d.h) best = min(best, max((int)col[(long long)(cy + dd) * d.w], dd));
  }
  clr[d.clr_off + (long long)cy * d.clr_ld + cx] = (uint8_t)(best == 0 ? 0 : max(1, best - 1));
}

// Sector skip planes (see MapDesc in sg_device.cuh).  Block (x, y): 256
// cells of the maps' concatenated cells, sector y.  The sector's offset list
// (cell offsets o with their skip J(o) = max(1, ceil(D(o) - 0.01)), sorted
// by the wedge distance D(o), every o with D(o) <= kSecRadius) is staged in
// shared memory; a free cell takes the J of the first offset whose cell is
// occupied or outside the map (the nearest obstacle in the widened sector),
// kSecRadius when there is none, and at least its Chebyshev skip.
__global__ void __launch_bounds__(256) k_sector_skip(const uint32_t* __restrict__ atlas, const uint8_t* __restrict__ clr,
                                                     const MapDesc* __restrict__ maps,
                                                     const long long* __restrict__ cell_prefix, int n_maps,
                                                     long long total, const uint32_t* __restrict__ table,
                                                     const int* __restrict__ tab_start, uint8_t* __restrict__ sec) {
  extern __shared__ uint32_t offs[];
  const int sector = blockIdx.y;
  const int t0 = tab_start[sector], nt = tab_start[sector + 1] - t0;
  for (int i = threadIdx.x; i < nt; i += blockDim.x) offs[i] = table[t0 + i];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const int m = find_map(cell_prefix, n_maps, i);
  const MapDesc d = maps[m];
  const long long local = i - cell_prefix[m];
  const int cx = (int)(local % d.w), cy = (int)(local / d.w);
  const int own = clr[d.clr_off + (long long)cy * d.clr_ld + cx];
  if (own == 0) return;  // occupied: the plane keeps its 0
  const uint32_t* rows = atlas + d.word_off;
  int J = kSecRadius;
  for (int e = 0; e < nt; ++e) {
    const uint32_t v = offs[e];
    const int px = cx + (int)(int8_t)(v & 0xFFu), py = cy + (int)(int8_t)((v >> 8) & 0xFFu);
    const bool blocked = (unsigned)px >= (unsigned)d.w || (unsigned)py >= (unsigned)d.h ||
                         ((rows[(long long)py * d.row_words + (px >> 5)] >> (px & 31)) & 1u);
    if (blocked) {
      J = (int)((v >> 16) & 0xFFu);
      break;
    }
  }
  sec[d.sec_off + (long long)sector * d.sec_plane + (long long)cy * d.clr_ld + cx] = (uint8_t)max(J, own);
}

// Episode 0 of every env; one warp per env.
template <bool kDyn>
__global__ void __launch_bounds__(128) k_reset(const __grid_constant__ DevCfg c, SimPtrs p, float* __restrict__ obs) {
  const int env = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (env >= c.n_envs) return;
  const EnvConst k = env_const(c, p, env, lane);
  Env s;
  s.t = 0;
  Obst b = {0.0f, 0.0f, 0.0f, 0.0f};
  Discs d;
  reset_env<kDyn>(c, k, s, 0u, lane, &b, &d);
  const Noise z = noise_for(k, s.sigma, s.ep_id, 0u, lane);
  ObsRegs o;
  Aux aux;
  observe<kDyn>(c, k, s, z, lane, o, aux, &d);
  if (obs) write_obs(obs + (long long)env * c.obs_dim, o, c.B, lane);
  if (lane == 0) store_env(p, env, s);
  if (kDyn && lane < c.n_dyn) store_obst(p, lane, env, b);
}

// One vectorized step of every env (sg_sim_step).  A warp takes kE
// envs (consecutive in the env order grouped by map): its lanes 0.. run the
// scalar part of the step for one env each (lane_step: state load, delay,
// Eq. 5, Eq. 6, collision, arrival, truncation, AutoReset draws and the
// scan-free terms of the observation and of Eq. 11, into shared records),
// then the whole warp scans each of its envs (lane j marches beam j): the
// post-motion state always (the observation, or the terminal observation and
// the reward of a done env), the reset state of a done env.  No warp waits on
// another.  Every value is the one-env-per-warp step's, in the same float32
// expressions.  kE envs per warp (6, 7 or 8; the host takes the count whose
// grid fills its last wave of resident CTAs best: at 65,536 envs 7, 70.8 us
// per launch, against 72.7 us with 8 and 77 us with 6; 4 per warp 75 us, 16
// per warp 75 us; 4 or 16 warps per CTA instead of 8 slower).
constexpr int kStepWarps = 8;

// Disc centres of an env for its two scans (dynamic obstacles only).
struct DiscRec {
  Discs a, b;
};

template <bool kDyn, int kE>
__global__ void __launch_bounds__(32 * kStepWarps, 4) k_step(const __grid_constant__ DevCfg c, SimPtrs p,
                                                             const int* __restrict__ order,
                                                             const uint8_t* __restrict__ act,
                                                             float* __restrict__ obs, float* __restrict__ rew,
                                                             uint8_t* __restrict__ done, float* __restrict__ term) {
  __shared__ StepScanRec rec[kStepWarps][kE];
  __shared__ DiscRec drec[kDyn ? kStepWarps : 1][kDyn ? kE : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int base = (blockIdx.x * kStepWarps + warp) * kE;
  if (base >= c.n_envs) return;  // warp-uniform
  const int nv = min(kE, c.n_envs - base);
  const bool live = lane < nv;
  const int i = live ? order[base + lane] : 0;
  Env s;
  if (live) s = load_env(p, i);
  // lanes past the warp's envs take part in the warp-wide collision tests only
  DiscRec* dr = kDyn ? &drec[warp][live ? lane : 0] : nullptr;
  const uint32_t d = lane_step<kDyn>(c, p, i, live, s, live ? (uint32_t)act[i] : 0u, rec[warp][live ? lane : 0],
                                     lane, kDyn ? &dr->a : nullptr, kDyn ? &dr->b : nullptr);
  if (live) {
    store_env(p, i, s);
    done[i] = (uint8_t)d;
  }
  __syncwarp();
  for (int e = 0; e < nv; ++e) {
    const StepScanRec& r = rec[warp][e];
    const int ie = r.env;
    const MapDesc m = p.maps[r.map];
    const uint32_t de = r.done;
    float b0, b1;
    const DiscRec* de_ = kDyn ? &drec[warp][e] : nullptr;
    const float mn = scan_env<kDyn, true>(c, p, m, r.nb, r.stepb, r.ax, r.ay, r.aphi, r.asigma,
                                    ((uint64_t)r.anhi << 32) | r.anlo, lane, b0, b1, kDyn ? &de_->a : nullptr);
    float rw;
    if (de & 1u)
      rw = -10.0f;
    else if (de & 2u)
      rw = 75.0f;
    else
      rw = reward_finish(c, r.rpart, mn);
    if (!de) {
      write_row(obs + (long long)ie * c.obs_dim, b0, b1, r.exa, c.B, lane);
    } else {
      if (term) write_row(term + (long long)ie * c.obs_dim, b0, b1, r.exa, c.B, lane);
      scan_env<kDyn, true>(c, p, m, r.nb, r.stepb, r.bx, r.by, r.bphi, r.bsigma, ((uint64_t)r.bnhi << 32) | r.bnlo, lane,
                     b0, b1, kDyn ? &de_->b : nullptr);
      write_row(obs + (long long)ie * c.obs_dim, b0, b1, r.exb, c.B, lane);
    }
    if (lane == 0) rew[ie] = rw;
  }
}

// K steps of one env with uniformly random actions drawn on the device; the
// env (and, with kDyn, its discs: lane o holds disc o) stays in registers
// between steps.  Per-step outputs are optional: obs_seq [K][n][obs_dim],
// act/rew/done_seq [K][n].
template <bool kDyn>
__device__ __forceinline__ void rollout_env(const DevCfg& c, const SimPtrs& p, int env, int lane, int K,
                                            float* __restrict__ obs, float* __restrict__ obs_seq,
                                            uint8_t* __restrict__ act_seq, float* __restrict__ rew_seq,
                                            uint8_t* __restrict__ done_seq) {
  const EnvConst k = env_const(c, p, env, lane);
  Env s = load_env(p, env);
  Obst b = {0.0f, 0.0f, 0.0f, 0.0f};
  Discs dsc;
  if (kDyn && lane < c.n_dyn) b = load_obst(p, lane, env);
  const uint64_t akey = sm_at(sm_at(c.seed, kStreamAction), (uint64_t)env);
  ObsRegs o;
  o.b0 = o.b1 = o.ex = 0.0f;
  const long long n = c.n_envs;
  uint32_t abatch = 0;
  for (int i = 0; i < K; ++i) {
    if ((i & 31) == 0) abatch = random_action_for(c, akey, s.t + (uint32_t)lane);
    const uint32_t a = __shfl_sync(kFull, abatch, i & 31);
    const StepOut r = env_step<kDyn>(c, p, k, s, a, lane, o, nullptr, &b, &dsc);
    if (obs_seq) write_obs(obs_seq + ((long long)i * n + env) * c.obs_dim, o, c.B, lane);
    if (lane == 0) {
      if (act_seq) act_seq[i * n + env] = (uint8_t)a;
      if (rew_seq) rew_seq[i * n + env] = r.rew;
      if (done_seq) done_seq[i * n + env] = (uint8_t)r.done;
    }
  }
  if (obs) write_obs(obs + (long long)env * c.obs_dim, o, c.B, lane);
  if (lane == 0) store_env(p, env, s);
  if (kDyn && lane < c.n_dyn) store_obst(p, lane, env, b);
}

// K steps of one env shared by W warps: every warp replays the pose chain of
// every step (it never depends on the LiDAR when actions are random), and
// warp w computes the observation and reward of the steps i with
// i mod W == w.  All warps hold identical states; no synchronisation.
__device__ __forceinline__ void rollout_env_split(const DevCfg& c, const SimPtrs& p, int env, int w, int W, int lane,
                                                  int K, float* __restrict__ obs, float* __restrict__ obs_seq,
                                                  uint8_t* __restrict__ act_seq, float* __restrict__ rew_seq,
                                                  uint8_t* __restrict__ done_seq) {
  const EnvConst k = env_const(c, p, env, lane);
  Env s = load_env(p, env);
  Env pre;
  const uint64_t akey = sm_at(sm_at(c.seed, kStreamAction), (uint64_t)env);
  ObsRegs o;
  o.b0 = o.b1 = o.ex = 0.0f;
  const long long n = c.n_envs;
  uint32_t abatch = 0;
  int mine = w;  // next step this warp observes
  for (int i = 0; i < K; ++i) {
    if ((i & 31) == 0) abatch = random_action_for(c, akey, s.t + (uint32_t)lane);
    const uint32_t a = __shfl_sync(kFull, abatch, i & 31);
    const uint32_t done = pose_step(c, p, k, s, pre, a, lane, w == 0);
    if (i == mine) {
      mine += W;
      const float r = obs_step(c, k, s, pre, done, lane, o);
      if (obs_seq) write_obs(obs_seq + ((long long)i * n + env) * c.obs_dim, o, c.B, lane);
      if (lane == 0) {
        if (act_seq) act_seq[i * n + env] = (uint8_t)a;
        if (rew_seq) rew_seq[i * n + env] = r;
        if (done_seq) done_seq[i * n + env] = (uint8_t)done;
      }
    }
  }
  if (obs && (K - 1) % W == w) write_obs(obs + (long long)env * c.obs_dim, o, c.B, lane);
  if (w == 0 && lane == 0) store_env(p, env, s);
}

// Pipelined variant: per env, one pose warp computes the state chain of a
// chunk of kPipeChunk steps and, one lane per step, everything of those
// steps that does not need the scan (goal frame, atan2, the five observation
// extras, the scan-free terms of Eq. 11, the noise key) into a shared-memory
// record buffer, while the other P warps of the env compute the scans,
// observations and rewards of the previous chunk; once its chunk is written
// the pose warp joins them.  Steps are handed out through a shared counter,
// so no warp waits on another's share.  The 1 + P warps of an env meet at a
// named barrier once per chunk (double-buffered observation records).
constexpr int kPipeChunk = 32;

struct __align__(16) StepRec {
  Env post;        // the state the step ends in (reset when done)
  uint32_t a;      // the action taken
  Env pre;         // after the motion, before the reset (written for done steps only)
  uint32_t done;
};
static_assert(sizeof(StepRec) == 128, "step record is eight 16-byte words");

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}
// Arrive without waiting (the other side of a producer / consumer barrier);
// the fence orders this warp's shared-memory accesses before the arrival.
__device__ __forceinline__ void named_arrive(int id, int nthreads) {
  __threadfence_block();
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint32_t fbits(float f) { return __float_as_uint(f); }
__device__ __forceinline__ float bitsf(uint32_t u) { return __uint_as_float(u); }

// An Env and one extra word as four 16-byte words.
__device__ __forceinline__ void pack_env(uint4* d, const Env& q, uint32_t w) {
  d[0] = make_uint4(fbits(q.x), fbits(q.y), fbits(q.phi), fbits(q.vl));
  d[1] = make_uint4(fbits(q.va), fbits(q.dt), fbits(q.K), fbits(q.cap));
  d[2] = make_uint4(fbits(q.sigma), q.ep_step, q.ep_id, q.t);
  d[3] = make_uint4(q.fifo, fbits(q.sphi), fbits(q.cphi), w);
}
__device__ __forceinline__ Env unpack_env(const uint4* d) {
  const uint4 a = d[0], b = d[1], e = d[2], f = d[3];
  Env q;
  q.x = bitsf(a.x), q.y = bitsf(a.y), q.phi = bitsf(a.z), q.vl = bitsf(a.w);
  q.va = bitsf(b.x), q.dt = bitsf(b.y), q.K = bitsf(b.z), q.cap = bitsf(b.w);
  q.sigma = bitsf(e.x), q.ep_step = e.y, q.ep_id = e.z, q.t = e.w;
  q.fifo = f.x, q.sphi = bitsf(f.y), q.cphi = bitsf(f.z);
  return q;
}

// What the scan of one step still needs.
struct __align__(16) ObsRec {
  float x, y, phi, sigma;  // the state observed (after the step, reset when done)
  uint32_t nlo, nhi;       // its noise key
  float rpart;             // scan-free part of Eq. 11 (of the pre-reset state when truncated)
  uint32_t da;             // done | action << 8
  float ex[5];             // observation entries B .. B + 4
  float px, py, pphi;      // pre-reset state (truncated steps)
  float psigma;
  uint32_t pnlo, pnhi;
  uint32_t pad;
};
static_assert(sizeof(ObsRec) == 80, "observation record is five 16-byte words");

__device__ __forceinline__ uint64_t noise_key(const EnvConst& k, const Env& s) {
  return sm_at(k.nkey, ((uint64_t)s.ep_id << 32) | s.ep_step);
}

// Lane j: record j of the chunk from its step record.
__device__ __forceinline__ void derive_rec(const DevCfg& c, const EnvConst& k, const StepRec& r, ObsRec& o) {
  const Env s = r.post;
  const uint32_t done = r.done;
  const GoalFrame g = goal_frame(k.L, s);
  const uint64_t nk = noise_key(k, s);
  float e[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) e[q] = obs_extra(c, k.L, s, g, q);
  float rp = 0.0f;
  if (!done) rp = reward_partial(c, k.L, s, g.alpha, g.ddx, g.ddy);
  uint4* w = reinterpret_cast<uint4*>(&o);
  w[0] = make_uint4(fbits(s.x), fbits(s.y), fbits(s.phi), fbits(s.sigma));
  w[1] = make_uint4((uint32_t)nk, (uint32_t)(nk >> 32), fbits(rp), done | (r.a << 8));
  w[2] = make_uint4(fbits(e[0]), fbits(e[1]), fbits(e[2]), fbits(e[3]));
  if (done && !(done & 3u)) {
    // truncated only: the reward comes from the scan before the reset
    const Env q = r.pre;
    const GoalFrame gp = goal_frame(k.L, q);
    const uint64_t pk = noise_key(k, q);
    o.rpart = reward_partial(c, k.L, q, gp.alpha, gp.ddx, gp.ddy);
    w[3] = make_uint4(fbits(e[4]), fbits(q.x), fbits(q.y), fbits(q.phi));
    w[4] = make_uint4(fbits(q.sigma), (uint32_t)pk, (uint32_t)(pk >> 32), 0u);
  } else {
    o.ex[4] = e[4];
  }
}

// The scan of one pose by a whole warp: this lane's beams (with noise drawn
// from key nk when sigma > 0) into o.b0 / o.b1; returns the minimum
// noise-free range over all beams.
template <bool kDyn = false>
__device__ __forceinline__ float scan_pose(const DevCfg& c, const EnvConst& k, float x, float y, float phi,
                                           float sigma, uint64_t nk, int lane, ObsRegs& o, const Discs* d = nullptr) {
  float n0 = 0.0f, n1 = 0.0f;
  if (sigma > 0.0f) {
    n0 = box_muller(sm_at(nk, (uint64_t)lane));
    if (k.nb > 32) n1 = box_muller(sm_at(nk, (uint64_t)(lane + 32)));
  }
  float mn = c.range_max;
  o.b0 = lane < k.nb ? beam_at<kDyn>(c, k, x, y, phi, sigma, k.off0, n0, mn, d) : 1.0f;
  o.b1 = lane + 32 < k.nb ? beam_at<kDyn>(c, k, x, y, phi, sigma, k.off1, n1, mn, d) : 1.0f;
  // ranges are >= 0, so their bit patterns order like the values
  return __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(mn)));
}

// The motion (delay, Eq. 5, Eq. 6) of steps j0 .. n-1 from state s as if no
// episode ended, lane j taking what belongs to step j (actions in lane j of
// abatch).  Only the velocity / heading recurrences and the position sums run
// in step order (every lane the same); the delayed action, the target
// velocities, sin/cos of each step's heading and the Eq. 6 increments are
// lane-parallel.  Every value is the float32 expression of kinematics(),
// evaluated in the same order.  Lane j writes step j's post state (with its
// action) to buf[j].post and returns its position and episode step in mx,
// my, mep; bad is set in the lanes whose action index is out of range.
__device__ __forceinline__ void motion_run(const DevCfg& c, const Env& s, int j0, int n, uint32_t abatch,
                                           StepRec* buf, int lane, bool& bad, float& mx, float& my,
                                           uint32_t& mep) {
  const bool mine = lane >= j0 && lane < n;
  const uint32_t q0 = s.fifo & 0xFFu, q1 = (s.fifo >> 8) & 0xFFu, d = (s.fifo >> 16) & 0xFFu;
  const uint32_t a = abatch;
  // the actions one and two steps back: this run's, else the FIFO's
  const uint32_t up1 = __shfl_up_sync(kFull, a & 0xFFu, 1), up2 = __shfl_up_sync(kFull, a & 0xFFu, 2);
  const uint32_t am1 = lane - 1 >= j0 ? up1 : q0;
  const uint32_t am2 = lane - 2 >= j0 ? up2 : (lane - 1 == j0 ? q0 : q1);
  const uint32_t ahat = d == 0 ? a : (d == 1 ? am1 : am2);
  const uint32_t fifo = (a & 0xFFu) | (am1 << 8) | (d << 16);
  float vhl = 0.0f, vha = 0.0f;
  if (ahat < (uint32_t)c.n_actions) {
    vhl = c.av[ahat] * s.cap;
    vha = c.aw[ahat] * s.cap;
  }
  const float omk = 1.0f - s.K;
  const float pl = omk * vhl, pa = omk * vha;
  if (mine && a >= (uint32_t)c.n_actions) bad = true;
  // Eq. 5 and the heading part of Eq. 6, in step order
  float vl = s.vl, va = s.va, phi = s.phi;
  float jvl = 0.0f, jva = 0.0f, jphi = s.phi;
  for (int j = j0; j < n; ++j) {
    const float plj = __shfl_sync(kFull, pl, j), paj = __shfl_sync(kFull, pa, j);
    vl = s.K * vl + plj;
    va = s.K * va + paj;
    float ph = phi + s.dt * va;
    if (ph >= kPi)
      ph = ph - 2.0f * kPi;
    else if (ph < -kPi)
      ph = ph + 2.0f * kPi;
    phi = ph;
    if (lane == j) {
      jvl = vl;
      jva = va;
      jphi = phi;
    }
  }
  float sn = s.sphi, cs = s.cphi;
  if (mine) f_sincos(jphi, sn, cs);
  // the position part of Eq. 6 uses the heading before the step: step j0's
  // from s, step j's from lane j - 1
  const float cu = __shfl_up_sync(kFull, cs, 1), su = __shfl_up_sync(kFull, sn, 1);
  const float cprev = lane == j0 ? s.cphi : cu, sprev = lane == j0 ? s.sphi : su;
  const float tx = s.dt * (jvl * cprev), ty = s.dt * (jvl * sprev);
  float x = s.x, y = s.y, jx = s.x, jy = s.y;
  for (int j = j0; j < n; ++j) {
    x = x - __shfl_sync(kFull, tx, j);
    y = y - __shfl_sync(kFull, ty, j);
    if (lane == j) {
      jx = x;
      jy = y;
    }
  }
  const uint32_t steps = (uint32_t)(lane - j0 + 1);
  if (mine) {
    Env e = s;
    e.x = jx, e.y = jy, e.phi = jphi, e.vl = jvl, e.va = jva;
    e.ep_step = s.ep_step + steps, e.t = s.t + steps, e.fifo = fifo;
    e.sphi = sn, e.cphi = cs;
    pack_env(reinterpret_cast<uint4*>(&buf[lane].post), e, a);
  }
  mx = jx;
  my = jy;
  mep = s.ep_step + steps;
}

// The pose chain of one chunk (n <= 32 steps, actions in lane j of abatch)
// by one warp, into the records buf[0..n).  The motion of a step (delay,
// Eq. 5, Eq. 6) needs the previous state only, and an episode end changes
// the chain only through the reset.  So the warp runs the motion through the
// rest of the chunk as if no episode ended (lane j keeps the position of step
// j), tests all those steps at once (lane j: centre out of the map, clearance
// around the centre, arrival, truncation), runs the bit-row collision test of
// the steps that need it in order with the whole warp, and takes the first
// step that ends the episode: the steps before it stand, it is reset, and the
// chain runs again from the step after it.  Every value equals that of
// stepping one step at a time.  With kDyn the env's discs (lane o holds disc
// o; its state between chunks in dst) move along with the pose chain, their
// centres after step j go to dpost[j] (the new episode's for a done step,
// whose pre-reset centres go to dpre[j]), and lane j's tests include them.
template <bool kDyn = false>
__device__ __forceinline__ void pose_chunk(const DevCfg& c, const SimPtrs& p, const EnvConst& k, Env& s, int n,
                                           uint32_t abatch, StepRec* buf, int lane, Obst* dst = nullptr,
                                           Discs* dpost = nullptr, Discs* dpre = nullptr) {
  bool bad = false;
  int j0 = 0;
  Obst b = {0.0f, 0.0f, 0.0f, 0.0f};
  if (kDyn && lane < c.n_dyn) b = dst[lane];
  while (j0 < n) {
    Obst bq = b;
    float mx, my;
    uint32_t mep;
    motion_run(c, s, j0, n, abatch, buf, lane, bad, mx, my, mep);
    if (kDyn) {
      // the discs move with the episode's control interval
      if (lane < c.n_dyn)
        for (int j = j0; j < n; ++j) {
          dyn_move(c, k.m, k.clr, s.dt, bq);
          dpost[j].x[lane] = bq.x;
          dpost[j].y[lane] = bq.y;
        }
    }
    __syncwarp();
    uint32_t done = 0;
    bool slow = false;
    if (lane >= j0 && lane < n) {
      if (mx < 0.0f || my < 0.0f || mx >= (float)k.m.w || my >= (float)k.m.h) {
        done = 1u;
      } else {
        const int own = __ldg(k.clr + __float2int_rd(my) * k.m.clr_ld + __float2int_rd(mx));
        slow = own < c.clr_collide;
      }
      const float ddx = k.L.gx - mx, ddy = k.L.gy - my;
      if (fmaf(ddx, ddx, ddy * ddy) <= c.goal_r * c.goal_r) done |= 2u;
      if (mep >= (uint32_t)c.t_max) done |= 4u;
      if (kDyn)
        for (int o = 0; o < c.n_dyn; ++o) {
          const float dx = dpost[lane].x[o] - mx, dy = dpost[lane].y[o] - my;
          if (fmaf(dx, dx, dy * dy) <= c.dyn_rr2) done |= 1u;
        }
    }
    uint32_t donem = __ballot_sync(kFull, done != 0u);
    uint32_t slowm = __ballot_sync(kFull, slow);
    while (slowm) {
      const int j = __ffs(slowm) - 1;
      slowm &= slowm - 1u;
      if (donem & ((1u << j) - 1u)) break;  // an earlier step ends the episode
      const float xj = __shfl_sync(kFull, mx, j), yj = __shfl_sync(kFull, my, j);
      if (collide_rows_warp(c, k.m, k.rows, xj, yj, lane)) {
        if (lane == j) done |= 1u;
        donem |= 1u << j;
      }
    }
    const int d = donem ? __ffs(donem) - 1 : n;
    if (lane >= j0 && lane < d) buf[lane].done = 0u;
    if (d == n) {
      s = unpack_env(reinterpret_cast<const uint4*>(&buf[n - 1].post));
      b = bq;
      break;
    }
    // step d ends the episode: its record keeps the state before the reset
    const uint32_t dd = __shfl_sync(kFull, done, d);
    const uint32_t ad = __shfl_sync(kFull, abatch, d);
    __syncwarp();
    Env e = unpack_env(reinterpret_cast<const uint4*>(&buf[d].post));
    __syncwarp();
    if (lane == 0) pack_env(reinterpret_cast<uint4*>(&buf[d].pre), e, dd);
    if (kDyn) {
      Discs nd;
      if (lane < c.n_dyn) {
        dpre[d].x[lane] = dpost[d].x[lane];
        dpre[d].y[lane] = dpost[d].y[lane];
      }
      reset_env<true>(c, k, e, e.ep_id + 1u, lane, &b, &nd);
      if (lane < c.n_dyn) {
        dpost[d].x[lane] = b.x;
        dpost[d].y[lane] = b.y;
      }
      __syncwarp();
    } else {
      reset_env(c, k, e, e.ep_id + 1u, lane);
    }
    if (lane == 0) pack_env(reinterpret_cast<uint4*>(&buf[d].post), e, ad);
    s = e;
    j0 = d + 1;
  }
  if (kDyn && lane < c.n_dyn) dst[lane] = b;
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(p.status, 1u);
}

// Consume the observation records of one chunk (steps i0 .. i1-1) through
// the shared counter: scan, observation, reward, outputs.  With kDyn the
// scans see the recorded disc centres of each step (dpost; dpre for the
// pre-reset scan of a truncated step).
template <bool kDyn = false>
__device__ __forceinline__ void consume_chunk(const DevCfg& c, const EnvConst& k, const ObsRec* buf, unsigned* next,
                                              int i0, int i1, int K, int env, long long n, int lane, ObsRegs& o,
                                              bool& has_last, float* __restrict__ obs_seq,
                                              uint8_t* __restrict__ act_seq, float* __restrict__ rew_seq,
                                              uint8_t* __restrict__ done_seq, const Discs* dpost = nullptr,
                                              const Discs* dpre = nullptr) {
  for (;;) {
    unsigned r = 0;
    if (lane == 0) r = atomicAdd(next, 1u);
    const int i = i0 + (int)__shfl_sync(kFull, r, 0);
    if (i >= i1) break;
    const ObsRec& R = buf[i - i0];
    const uint32_t da = R.da, done = da & 0xFFu;
    float rew = 0.0f;
    if (done & 1u) {
      rew = -10.0f;
    } else if (done & 2u) {
      rew = 75.0f;
    } else if (done) {
      const uint64_t pk = ((uint64_t)R.pnhi << 32) | R.pnlo;
      rew = reward_finish(c, R.rpart, scan_pose<kDyn>(c, k, R.px, R.py, R.pphi, R.psigma, pk, lane, o,
                                                      kDyn ? dpre + (i - i0) : nullptr));
    }
    const uint64_t nk = ((uint64_t)R.nhi << 32) | R.nlo;
    const float mn = scan_pose<kDyn>(c, k, R.x, R.y, R.phi, R.sigma, nk, lane, o, kDyn ? dpost + (i - i0) : nullptr);
    if (!done) rew = reward_finish(c, R.rpart, mn);
    o.ex = lane < 5 ? R.ex[lane] : 0.0f;
    if (i == K - 1) has_last = true;
    if (obs_seq) write_obs(obs_seq + ((long long)i * n + env) * c.obs_dim, o, c.B, lane);
    if (lane == 0) {
      if (act_seq) act_seq[i * n + env] = (uint8_t)(da >> 8);
      if (rew_seq) rew_seq[i * n + env] = rew;
      if (done_seq) done_seq[i * n + env] = (uint8_t)done;
    }
  }
}

// Named barriers of env group g: full(b) = 1 + 4g + b (records of buffer b
// written: the pose warp arrives, the observation warps wait), free(b) =
// 3 + 4g + b (buffer b consumed: the observation warps arrive, the pose warp
// waits before writing it again).  At most kPipeMaxGroups groups per CTA.
constexpr int kPipeMaxGroups = 3;

// Shared memory of one env group of the pipelined kernel.
__host__ __device__ constexpr size_t pipe_group_bytes(bool dyn) {
  return kPipeChunk * (sizeof(StepRec) + 2 * sizeof(ObsRec)) +
         (dyn ? 4 * kPipeChunk * sizeof(Discs) + kMaxDyn * sizeof(Obst) : 0);
}
static_assert(pipe_group_bytes(false) % 16 == 0 && pipe_group_bytes(true) % 16 == 0, "16-byte aligned groups");

// Time slicing (seg > 0): the rollout is cut into segments of seg steps and
// a persistent grid takes work items (segment, CTA's envs) in segment-major
// order from a device counter, so that every resident CTA stays busy to the
// end instead of the last wave running part-empty.  An item starts after the
// previous segment of its envs has stored their state: its CTA waits on a
// per-envs flag (bounded; on timeout the status word gets SG_DEV_TIMEOUT, an
// abort word stops the other CTAs, and the launch's outputs are incomplete).
// sync: [nblk] flags (segments done), item counter, abort word; zero at launch.
constexpr unsigned kPipeWaitIters = 1u << 22;  // default bound, x ~256 ns sleeps: about a second

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned* a, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(a), "r"(v) : "memory");
}

// State of env i through L2 (another SM may have written it in this launch).
__device__ __forceinline__ Env load_env_cg(const SimPtrs& p, int i) {
  Env s;
  const int n = p.n;
  s.x = __ldcg(p.f + 0 * n + i);
  s.y = __ldcg(p.f + 1 * n + i);
  s.phi = __ldcg(p.f + 2 * n + i);
  s.vl = __ldcg(p.f + 3 * n + i);
  s.va = __ldcg(p.f + 4 * n + i);
  s.dt = __ldcg(p.f + 5 * n + i);
  s.K = __ldcg(p.f + 6 * n + i);
  s.cap = __ldcg(p.f + 7 * n + i);
  s.sigma = __ldcg(p.f + 8 * n + i);
  s.ep_step = __ldcg(p.u + 0 * n + i);
  s.ep_id = __ldcg(p.u + 1 * n + i);
  s.t = __ldcg(p.u + 2 * n + i);
  s.fifo = __ldcg(p.u + 3 * n + i);
  f_sincos(s.phi, s.sphi, s.cphi);
  return s;
}
__device__ __forceinline__ Obst load_obst_cg(const SimPtrs& p, int o, int i) {
  const int n = p.n;
  Obst b;
  b.x = __ldcg(p.dyn + (4 * o + 0) * n + i);
  b.y = __ldcg(p.dyn + (4 * o + 1) * n + i);
  b.vx = __ldcg(p.dyn + (4 * o + 2) * n + i);
  b.vy = __ldcg(p.dyn + (4 * o + 3) * n + i);
  return b;
}

template <bool kDyn>
__global__ void __launch_bounds__(512, 2) k_rollout_random_pipe(const __grid_constant__ DevCfg c, SimPtrs p, int K,
                                                                int P, const int* __restrict__ order, int seg,
                                                                unsigned* __restrict__ sync, unsigned wait_iters,
                                                                float* __restrict__ obs,
                                                                float* __restrict__ obs_seq,
                                                                uint8_t* __restrict__ act_seq,
                                                                float* __restrict__ rew_seq,
                                                                uint8_t* __restrict__ done_seq) {
  extern __shared__ __align__(16) unsigned char pipe_smem[];
  __shared__ unsigned next_step[kPipeMaxGroups][2];  // per env group and buffer: next record to take
  __shared__ int item_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = 1 + P;  // warps per env
  const int group = warp / G, role = warp % G;
  const int E = blockDim.x / (32 * G);
  const int nblk = (c.n_envs + E - 1) / E;
  const int seglen = seg > 0 ? seg : K;  // a multiple of kPipeChunk when seg > 0
  const int nseg = (K + seglen - 1) / seglen;
  const long long nitems = (long long)nblk * nseg;
  // per group: kPipeChunk step records, 2 x kPipeChunk observation records,
  // and with discs 2 x kPipeChunk centre sets after each step, 2 x kPipeChunk
  // before a reset, and the disc state between chunks
  unsigned char* base = pipe_smem + (size_t)group * pipe_group_bytes(kDyn);
  StepRec* st = reinterpret_cast<StepRec*>(base);
  ObsRec* ob = reinterpret_cast<ObsRec*>(base + kPipeChunk * sizeof(StepRec));
  Discs* dpost = reinterpret_cast<Discs*>(ob + 2 * kPipeChunk);
  Discs* dpre = dpost + 2 * kPipeChunk;
  Obst* dst = reinterpret_cast<Obst*>(dpre + 2 * kPipeChunk);
  const int bfull = 1 + 4 * group, bfree = 3 + 4 * group, nthr = 32 * G;
  const long long n = c.n_envs;
  for (int iter = 0;; ++iter) {
    // next item: its segment and CTA's envs, after the previous segment of
    // those envs is stored
    if (threadIdx.x == 0) {
      long long it;
      if (!sync)
        it = iter == 0 ? (long long)blockIdx.x : nitems;
      else
        it = __ldcg(&sync[nblk + 1]) ? nitems : (long long)atomicAdd(&sync[nblk], 1u);
      if (sync && it < nitems && it >= nblk) {
        const unsigned need = (unsigned)(it / nblk);
        unsigned w = 0;
        while (ld_acquire_gpu(&sync[it % nblk]) < need) {
          if (++w > wait_iters || ld_acquire_gpu(&sync[nblk + 1])) {
            atomicOr(p.status, SG_DEV_TIMEOUT);
            atomicExch(&sync[nblk + 1], 1u);
            it = nitems;
            break;
          }
          __nanosleep(256);
        }
      }
      item_sh = it < nitems ? (int)it : -1;
    }
    __syncthreads();
    const int item = item_sh;
    __syncthreads();  // item_sh is rewritten by the next iteration
    if (item < 0) break;
    const int blk = item % nblk, sg_i = item / nblk;
    const int s0 = sg_i * seglen, s1 = min(K, s0 + seglen), Kl = s1 - s0;
    const int slot = blk * E + group;
    if (slot < c.n_envs) {  // the whole group takes part or not
      const int env = order ? order[slot] : slot;
      const EnvConst k = env_const(c, p, env, lane);
      const int chunks = (Kl + kPipeChunk - 1) / kPipeChunk;
      ObsRegs o;
      o.b0 = o.b1 = o.ex = 0.0f;
      bool has_last = false;
      if (role == 0) {
        for (int ch = 0; ch <= chunks; ++ch) {
          if (ch < chunks) {
            const int b = ch & 1;
            if (ch >= 2) named_barrier(bfree + b, nthr);  // chunk ch - 2 consumed
            if (lane == 0) next_step[group][b] = 0u;
            // the state carried between chunks is the last step record's post
            // state, so nothing of the pose chain stays live while this warp
            // takes observation records
            Env s = ch > 0 ? unpack_env(reinterpret_cast<const uint4*>(&st[kPipeChunk - 1].post))
                           : (sync ? load_env_cg(p, env) : load_env(p, env));
            if (kDyn && ch == 0 && lane < c.n_dyn) dst[lane] = sync ? load_obst_cg(p, lane, env) : load_obst(p, lane, env);
            const int i0 = ch * kPipeChunk, nst = min(Kl, i0 + kPipeChunk) - i0;
            // lane l draws the action of step i0 + l (t counts every step)
            const uint64_t akey = sm_at(sm_at(c.seed, kStreamAction), (uint64_t)env);
            const uint32_t abatch = random_action_for(c, akey, s.t + (uint32_t)lane);
            pose_chunk<kDyn>(c, p, k, s, nst, abatch, st, lane, dst, dpost + b * kPipeChunk,
                             dpre + b * kPipeChunk);
            __syncwarp();
            if (lane < nst) derive_rec(c, k, st[lane], ob[b * kPipeChunk + lane]);
            named_arrive(bfull + b, nthr);
          }
          if (ch >= 1) {
            const int b = (ch - 1) & 1, i0 = s0 + (ch - 1) * kPipeChunk;
            consume_chunk<kDyn>(c, k, ob + b * kPipeChunk, &next_step[group][b], i0, min(s1, i0 + kPipeChunk), K,
                                env, n, lane, o, has_last, obs_seq, act_seq, rew_seq, done_seq,
                                dpost + b * kPipeChunk, dpre + b * kPipeChunk);
          }
        }
        // the last two chunks' consumption completes the free barriers' phases
        for (int ch = max(chunks, 2); ch < chunks + 2; ++ch) named_barrier(bfree + (ch & 1), nthr);
        if (lane == 0 && chunks > 0)
          store_env(p, env, unpack_env(reinterpret_cast<const uint4*>(&st[Kl - 1 - (chunks - 1) * kPipeChunk].post)));
        if (kDyn && lane < c.n_dyn) store_obst(p, lane, env, dst[lane]);
        if (sync) __threadfence();
      } else {
        for (int ch = 1; ch <= chunks; ++ch) {
          const int b = (ch - 1) & 1, i0 = s0 + (ch - 1) * kPipeChunk;
          named_barrier(bfull + b, nthr);  // chunk ch - 1 written
          consume_chunk<kDyn>(c, k, ob + b * kPipeChunk, &next_step[group][b], i0, min(s1, i0 + kPipeChunk), K, env,
                              n, lane, o, has_last, obs_seq, act_seq, rew_seq, done_seq, dpost + b * kPipeChunk,
                              dpre + b * kPipeChunk);
          named_arrive(bfree + b, nthr);
        }
      }
      if (obs && has_last) write_obs(obs + (long long)env * c.obs_dim, o, c.B, lane);
    }
    if (!sync) break;
    // every group's state is stored: publish this segment of the CTA's envs
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release_gpu(&sync[blk], (unsigned)(sg_i + 1));
    }
  }
}

static size_t pipe_smem_bytes(int E, bool dyn) { return (size_t)E * pipe_group_bytes(dyn); }
static int pipe_envs_per_block(const sg_launch& L) {
  const int E = L.warps_per_block / (1 + L.obs_warps);
  return E < 1 ? 1 : (E > kPipeMaxGroups ? kPipeMaxGroups : E);
}


// W warps per env, E envs per CTA (blockDim = 32 W E).
__global__ void __launch_bounds__(256, 4) k_rollout_random_split(const __grid_constant__ DevCfg c, SimPtrs p, int K,
                                                              int W, float* __restrict__ obs,
                                                              float* __restrict__ obs_seq,
                                                              uint8_t* __restrict__ act_seq,
                                                              float* __restrict__ rew_seq,
                                                              uint8_t* __restrict__ done_seq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int env = blockIdx.x * (blockDim.x / (32 * W)) + warp / W;
  if (env >= c.n_envs) return;
  rollout_env_split(c, p, env, warp % W, W, lane, K, obs, obs_seq, act_seq, rew_seq, done_seq);
}

// One warp per env, envs in index order.
template <bool kDyn>
__global__ void __launch_bounds__(512, 2) k_rollout_random(const __grid_constant__ DevCfg c, SimPtrs p, int K,
                                                        float* __restrict__ obs, float* __restrict__ obs_seq,
                                                        uint8_t* __restrict__ act_seq, float* __restrict__ rew_seq,
                                                        uint8_t* __restrict__ done_seq) {
  const int env = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (env >= c.n_envs) return;
  rollout_env<kDyn>(c, p, env, lane, K, obs, obs_seq, act_seq, rew_seq, done_seq);
}

// Persistent variant for uneven batches: a fixed grid of warps pulls envs
// from a work list (typically sorted by cost, longest first) through a
// device counter, so that envs with many beams or large maps start first and
// short ones fill the tail.
template <bool kDyn>
__global__ void __launch_bounds__(512, 2) k_rollout_random_queue(const __grid_constant__ DevCfg c, SimPtrs p, int K,
                                                              const int* __restrict__ order,
                                                              unsigned* __restrict__ next, float* __restrict__ obs,
                                                              float* __restrict__ obs_seq, uint8_t* __restrict__ act_seq,
                                                              float* __restrict__ rew_seq,
                                                              uint8_t* __restrict__ done_seq) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned w = 0;
    if (lane == 0) w = atomicAdd(next, 1u);
    w = __shfl_sync(kFull, w, 0);
    if (w >= (unsigned)c.n_envs) break;
    const int env = order ? order[w] : (int)w;
    rollout_env<kDyn>(c, p, env, lane, K, obs, obs_seq, act_seq, rew_seq, done_seq);
  }
}

// ------------------------------------------------------------- host side

namespace {
thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char* what) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
  return SG_E_CUDA;
}
#define SG_CUDA(call)                                           \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);         \
  } while (0)

constexpr int kWarpsPerBlock = 4;

int grid_for(int n_envs) { return (n_envs + kWarpsPerBlock - 1) / kWarpsPerBlock; }

// Host-side cost of an env for the work list: beams x the march work one
// beam of its map can take (clearance-skipped march: about proportional to
// the number of beams; larger maps are less cache friendly).
double env_cost(int beams, int w, int h) { return (double)beams * (1.0 + 1e-6 * (double)w * (double)h); }

bool finite_nonneg(float v) { return std::isfinite(v) && v >= 0.0f; }
}  // namespace

const char* sg_cuda_err_text() { return g_cuda_err; }
int sg_set_cuda_error(cudaError_t e, const char* what) { return cuda_fail(e, what); }
int sg_set_error_text(const char* msg, int code) {
  std::snprintf(g_cuda_err, sizeof(g_cuda_err), "%s", msg);
  return code;
}

// Validates the configuration; fills the launch-time copy.
static int make_devcfg(const sg_sim_config* cfg, DevCfg* dc) {
  if (cfg->n_envs < 1 || cfg->n_envs > (1 << 24)) return SG_E_INVAL;
  if (cfg->n_beams < 2 || cfg->n_beams > 64) return SG_E_INVAL;
  if (cfg->n_actions < 1 || cfg->n_actions > 8) return SG_E_INVAL;
  if (cfg->t_max < 1) return SG_E_INVAL;
  if (cfg->delay_lo < 0 || cfg->delay_hi > 2 || cfg->delay_lo > cfg->delay_hi) return SG_E_INVAL;
  if (!(cfg->range_max > 0.0f) || !(cfg->march_step > 0.0f) || !std::isfinite(cfg->range_max)) return SG_E_INVAL;
  const float kmaxf = std::floor(cfg->range_max / cfg->march_step);
  if (!(kmaxf >= 1.0f) || kmaxf > 4096.0f) return SG_E_INVAL;
  if (!finite_nonneg(cfg->fov) || !finite_nonneg(cfg->robot_radius) || !finite_nonneg(cfg->goal_radius))
    return SG_E_INVAL;
  if (cfg->fov > 6.2831855f) return SG_E_INVAL;  // at most one turn
  if (cfg->march_sectors < 0 || cfg->march_sectors > kMaxSectors ||
      (cfg->march_sectors > 1 && (cfg->march_sectors & (cfg->march_sectors - 1))) || cfg->march_sectors == 2)
    return SG_E_INVAL;
  if (!std::isfinite(cfg->near_dist) || !std::isfinite(cfg->start_offset) || !finite_nonneg(cfg->start_jitter))
    return SG_E_INVAL;
  const float pairs[][2] = {{cfg->dt_lo, cfg->dt_hi}, {cfg->k_lo, cfg->k_hi}, {cfg->cap_lo, cfg->cap_hi},
                            {cfg->sigma_lo, cfg->sigma_hi}};
  for (const auto& pr : pairs)
    if (!std::isfinite(pr[0]) || !std::isfinite(pr[1]) || pr[0] > pr[1]) return SG_E_INVAL;
  if (cfg->sigma_lo < 0.0f) return SG_E_INVAL;
  if (!(cfg->v_nom > 0.0f) || !(cfg->w_nom > 0.0f)) return SG_E_INVAL;
  if (cfg->n_dyn < 0 || cfg->n_dyn > kMaxDyn) return SG_E_INVAL;
  if (cfg->n_dyn > 0) {
    if (!(cfg->dyn_radius > 0.0f) || !std::isfinite(cfg->dyn_radius)) return SG_E_INVAL;
    if (!finite_nonneg(cfg->dyn_speed_lo) || !std::isfinite(cfg->dyn_speed_hi) ||
        cfg->dyn_speed_lo > cfg->dyn_speed_hi || !finite_nonneg(cfg->dyn_keepout))
      return SG_E_INVAL;
  }
  std::memset(dc, 0, sizeof(*dc));
  dc->n_envs = cfg->n_envs;
  dc->B = cfg->n_beams;
  dc->obs_dim = cfg->n_beams + 5;
  dc->n_actions = cfg->n_actions;
  dc->t_max = cfg->t_max;
  dc->kmax = (int)kmaxf;
  dc->delay_lo = cfg->delay_lo;
  dc->delay_span = cfg->delay_hi - cfg->delay_lo + 1;
  dc->skip_ok = cfg->march_step <= 1.0f ? 1 : 0;
  // a point of a cell with clearance c is at least c - 0.5 cells from every
  // occupied cell centre; keep a margin of one cell above the radius so that
  // the rounded disc test could not have fired either
  dc->clr_collide = (int)std::ceil(cfg->robot_radius) + 1;
  dc->fov = cfg->fov;
  dc->half_fov = cfg->fov * 0.5f;
  dc->range_max = cfg->range_max;
  dc->delta = cfg->march_step;
  dc->robot_r = cfg->robot_radius;
  dc->goal_r = cfg->goal_radius;
  dc->near_dist = cfg->near_dist;
  dc->start_offset = cfg->start_offset;
  dc->jitter = cfg->start_jitter;
  dc->dt_lo = cfg->dt_lo;
  dc->dt_hi = cfg->dt_hi;
  dc->k_lo = cfg->k_lo;
  dc->k_hi = cfg->k_hi;
  dc->cap_lo = cfg->cap_lo;
  dc->cap_hi = cfg->cap_hi;
  dc->sig_lo = cfg->sigma_lo;
  dc->sig_hi = cfg->sigma_hi;
  dc->v_nom = cfg->v_nom;
  dc->w_nom = cfg->w_nom;
  for (int i = 0; i < 8; ++i) {
    dc->av[i] = cfg->action_v[i];
    dc->aw[i] = cfg->action_w[i];
  }
  dc->seed = cfg->seed;
  dc->n_dyn = cfg->n_dyn;
  if (cfg->n_dyn > 0) {
    // float32 products, as the step evaluates them
    const float r = cfg->dyn_radius, rr = cfg->robot_radius + cfg->dyn_radius, kp = cfg->dyn_keepout;
    dc->dyn_r = r;
    dc->dyn_r2 = r * r;
    dc->dyn_rr2 = rr * rr;
    dc->dyn_keep2 = kp * kp;
    dc->dyn_vlo = cfg->dyn_speed_lo;
    dc->dyn_vhi = cfg->dyn_speed_hi;
    dc->dyn_re = r + cfg->march_step + 0.25f;
  }
  return SG_OK;
}

// ---------------------------------------------------- sector skip tables
// Wedge distance of a cell offset o for the direction sector [a0, a1]
// (a1 - a0 < pi): the smallest |w| over the points w of the square
// [ox - 1, ox + 1] x [oy - 1, oy + 1] (every difference q' - q of a point q'
// of the offset cell and a point q of the origin cell) whose direction lies
// in the sector; infinity when only w = 0 does (no forward motion within the
// sector reaches the cell).  The square is clipped by the sector's two
// bounding half-planes (Sutherland-Hodgman), then the distance from the
// origin to the convex remainder is taken.
static int clip_halfplane(const double (*in)[2], int n, double nx, double ny, double (*out)[2]) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const double* P = in[i];
    const double* Q = in[(i + 1) % n];
    const double dp = nx * P[0] + ny * P[1], dq = nx * Q[0] + ny * Q[1];
    if (dp >= 0.0) {
      out[m][0] = P[0];
      out[m][1] = P[1];
      ++m;
    }
    if ((dp >= 0.0) != (dq >= 0.0)) {
      const double t = dp / (dp - dq);
      out[m][0] = P[0] + t * (Q[0] - P[0]);
      out[m][1] = P[1] + t * (Q[1] - P[1]);
      ++m;
    }
  }
  return m;
}

static double segment_to_origin(const double* A, const double* B) {
  const double dx = B[0] - A[0], dy = B[1] - A[1];
  const double L = dx * dx + dy * dy;
  double t = L > 0.0 ? -(A[0] * dx + A[1] * dy) / L : 0.0;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const double px = A[0] + t * dx, py = A[1] + t * dy;
  return std::sqrt(px * px + py * py);
}

double sg_wedge_distance(int ox, int oy, double a0, double a1) {
  double sq[4][2] = {{ox - 1.0, oy - 1.0}, {ox + 1.0, oy - 1.0}, {ox + 1.0, oy + 1.0}, {ox - 1.0, oy + 1.0}};
  double t1[16][2], t2[16][2];
  // left of the ray at a0 and right of the ray at a1
  int n = clip_halfplane(sq, 4, -std::sin(a0), std::cos(a0), t1);
  if (n == 0) return HUGE_VAL;
  n = clip_halfplane(t1, n, std::sin(a1), -std::cos(a1), t2);
  if (n == 0) return HUGE_VAL;
  double far = 0.0;
  for (int i = 0; i < n; ++i) far = std::max(far, std::hypot(t2[i][0], t2[i][1]));
  if (far < 1e-9) return HUGE_VAL;  // the apex alone
  bool inside = true;  // the origin inside the (counter-clockwise) polygon
  for (int i = 0; i < n && inside; ++i) {
    const double* P = t2[i];
    const double* Q = t2[(i + 1) % n];
    if ((Q[0] - P[0]) * (-P[1]) - (Q[1] - P[1]) * (-P[0]) < -1e-12) inside = false;
  }
  if (inside) return 0.0;
  double best = HUGE_VAL;
  for (int i = 0; i < n; ++i) best = std::min(best, segment_to_origin(t2[i], t2[(i + 1) % n]));
  return best;
}

// Offset lists of the n_sec sectors: entry = ox & 0xFF | (oy & 0xFF) << 8 |
// J << 16 with J = max(1, ceil(D - 0.01)), sorted by D (then oy, ox), every
// offset with D <= kSecRadius; start[s] .. start[s + 1] is sector s.
constexpr double kSecWiden = 0.01;   // radians added on both sides of a sector
constexpr double kSecMargin = 0.01;  // cells taken off the wedge distance

void sg_sector_table(int n_sec, std::vector<uint32_t>& table, std::vector<int>& start) {
  table.clear();
  start.assign(1, 0);
  const int R = kSecRadius + 2;
  struct E {
    double d;
    int ox, oy;
  };
  std::vector<E> list;
  for (int sct = 0; sct < n_sec; ++sct) {
    const double a0 = -M_PI + sct * 2.0 * M_PI / n_sec - kSecWiden;
    const double a1 = -M_PI + (sct + 1) * 2.0 * M_PI / n_sec + kSecWiden;
    list.clear();
    for (int oy = -R; oy <= R; ++oy)
      for (int ox = -R; ox <= R; ++ox) {
        if (ox == 0 && oy == 0) continue;  // the cell the sample is in (free)
        const double d = sg_wedge_distance(ox, oy, a0, a1);
        if (d <= (double)kSecRadius) list.push_back({d, ox, oy});
      }
    std::sort(list.begin(), list.end(), [](const E& a, const E& b) {
      return a.d != b.d ? a.d < b.d : (a.oy != b.oy ? a.oy < b.oy : a.ox < b.ox);
    });
    for (const E& e : list) {
      const int J = std::max(1, (int)std::ceil(e.d - kSecMargin));
      table.push_back((uint32_t)(e.ox & 0xFF) | ((uint32_t)(e.oy & 0xFF) << 8) | ((uint32_t)J << 16));
    }
    start.push_back((int)table.size());
  }
}

// Build the sector planes of every map (the skip maps and bit atlas exist).
static cudaError_t build_sector_planes(sg_sim* s) {
  std::vector<uint32_t> table;
  std::vector<int> start;
  sg_sector_table(s->dc.n_sec, table, start);
  int max_list = 0;
  for (int i = 0; i < s->dc.n_sec; ++i) max_list = std::max(max_list, start[i + 1] - start[i]);
  std::vector<long long> prefix((size_t)s->n_maps + 1, 0);
  for (int m = 0; m < s->n_maps; ++m)
    prefix[m + 1] = prefix[m] + (long long)s->maps_host[m].w * s->maps_host[m].h;
  uint32_t* tab_dev = nullptr;
  int* start_dev = nullptr;
  long long* prefix_dev = nullptr;
  cudaError_t e = cudaMalloc((void**)&tab_dev, table.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&start_dev, start.size() * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&prefix_dev, prefix.size() * 8);
  if (e == cudaSuccess) e = cudaMemcpy(tab_dev, table.data(), table.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(start_dev, start.data(), start.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(prefix_dev, prefix.data(), prefix.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->sec, 0, (size_t)s->sec_bytes);  // zero borders and occupied cells
  if (e == cudaSuccess) {
    const size_t smem = (size_t)max_list * 4;
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(k_sector_skip, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const long long total = prefix.back();
    if (e == cudaSuccess) {
      dim3 grid((unsigned)((total + 255) / 256), (unsigned)s->dc.n_sec);
      k_sector_skip<<<grid, 256, smem>>>(s->atlas, s->clr, s->maps_dev, prefix_dev, s->n_maps, total, tab_dev,
                                         start_dev, s->sec);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(tab_dev);
  cudaFree(start_dev);
  cudaFree(prefix_dev);
  return e;
}

SimPtrs sg_sim_ptrs(sg_sim* s) {
  SimPtrs p;
  p.f = s->fstate;
  p.u = s->ustate;
  p.atlas = s->atlas;
  p.clr = s->clr;
  p.sec = s->sec;
  p.maps = s->maps_dev;
  p.env_map = s->env_map_dev;
  p.env_beams = s->env_beams_dev;
  p.status = s->status_dev;
  p.dyn = s->dyn;
  p.n = s->dc.n_envs;
  p.pad = 0;
  return p;
}

static void free_sim(sg_sim* s) {
  if (!s) return;
  cudaFree(s->atlas);
  cudaFree(s->clr);
  cudaFree(s->sec);
  cudaFree(s->maps_dev);
  cudaFree(s->env_map_dev);
  cudaFree(s->env_beams_dev);
  cudaFree(s->fstate);
  cudaFree(s->ustate);
  cudaFree(s->status_dev);
  cudaFree(s->order_dev);
  cudaFree(s->queue_dev);
  cudaFree(s->map_order_dev);
  cudaFree(s->dyn);
  cudaFree(s->pipe_sync_dev);
  cudaFree(s->q_sync_dev);
  delete s;
}

extern "C" int sg_sim_create(const sg_sim_config* cfg, int32_t n_maps, const uint8_t* const* maps_host,
                             const int32_t* map_w, const int32_t* map_h, const int32_t* env_map,
                             const int32_t* env_beams, sg_sim_t* out) {
  SG_RANGE("sg_sim_create");
  if (!cfg || !maps_host || !map_w || !map_h || !env_map || !out) return SG_E_INVAL;
  if (n_maps < 1) return SG_E_INVAL;
  *out = nullptr;
  DevCfg dc;
  int rc = make_devcfg(cfg, &dc);
  if (rc) return rc;
  const int n = cfg->n_envs;
  std::vector<MapDesc> md((size_t)n_maps);
  long long words = 0;
  long long clr_bytes = 0;
  size_t max_cells = 0;
  for (int m = 0; m < n_maps; ++m) {
    if (!maps_host[m] || map_w[m] < 1 || map_h[m] < 1 || map_w[m] > 16384 || map_h[m] > 16384) return SG_E_INVAL;
    // a disc must fit between the walls: r_o < W - r_o (in float32)
    if (cfg->n_dyn > 0 && !((float)map_w[m] - cfg->dyn_radius > cfg->dyn_radius &&
                            (float)map_h[m] - cfg->dyn_radius > cfg->dyn_radius))
      return SG_E_INVAL;
    md[m].word_off = words;
    md[m].w = map_w[m];
    md[m].h = map_h[m];
    md[m].row_words = ((map_w[m] + 127) / 128) * 4;  // rows padded to 16 bytes
    md[m].clr_ld = map_w[m] + 2 * kClrBorder;
    md[m].clr_off = clr_bytes + (long long)kClrBorder * md[m].clr_ld + kClrBorder;
    words += (long long)md[m].row_words * map_h[m];
    clr_bytes += (long long)md[m].clr_ld * (map_h[m] + 2 * kClrBorder);
    max_cells = std::max(max_cells, (size_t)map_w[m] * (size_t)map_h[m]);
  }
  for (int i = 0; i < n; ++i) {
    if (env_map[i] < 0 || env_map[i] >= n_maps) return SG_E_INVAL;
    if (env_beams && (env_beams[i] < 2 || env_beams[i] > cfg->n_beams)) return SG_E_INVAL;
  }
  // sector skip planes: n_sec planes of the skip-map layout per map
  int n_sec = dc.skip_ok ? cfg->march_sectors : 1;
  if (n_sec == 0) {
    // 16 sectors while the planes fit in L2 (there they halve the march's
    // iterations; streamed from DRAM they cost more than they save), else
    // the Chebyshev skip map alone
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
      l2 = 0;
    n_sec = 16.0 * (double)clr_bytes <= (double)l2 ? 16 : 1;
  }
  dc.n_sec = n_sec;
  dc.sec_scale = (float)((double)n_sec / (2.0 * M_PI));
  long long sec_bytes = 0;
  for (int m = 0; m < n_maps; ++m) {
    const long long plane = (long long)md[m].clr_ld * (map_h[m] + 2 * kClrBorder);
    md[m].sec_plane = n_sec > 1 ? plane : 0;
    md[m].sec_off = n_sec > 1 ? sec_bytes + (long long)kClrBorder * md[m].clr_ld + kClrBorder : 0;
    if (n_sec > 1) sec_bytes += plane * n_sec;
  }
  sg_sim* s = new (std::nothrow) sg_sim();
  if (!s) return SG_E_OOM;
  s->cfg = *cfg;
  s->dc = dc;
  s->n_maps = n_maps;
  s->maps_host = md;
  s->atlas_words = words;
  s->clr_bytes = clr_bytes;
  s->sec_bytes = sec_bytes;
  cudaGetDevice(&s->device);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** ptr, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(ptr, bytes);
  };
  alloc((void**)&s->atlas, (size_t)words * 4);
  alloc((void**)&s->clr, (size_t)clr_bytes);
  if (sec_bytes > 0) alloc((void**)&s->sec, (size_t)sec_bytes);
  alloc((void**)&s->maps_dev, sizeof(MapDesc) * n_maps);
  alloc((void**)&s->env_map_dev, sizeof(int) * n);
  if (env_beams) alloc((void**)&s->env_beams_dev, sizeof(int) * n);
  alloc((void**)&s->fstate, sizeof(float) * 9 * (size_t)n);
  alloc((void**)&s->ustate, sizeof(uint32_t) * 4 * (size_t)n);
  alloc((void**)&s->status_dev, sizeof(uint32_t));
  alloc((void**)&s->map_order_dev, sizeof(int) * n);
  if (cfg->n_dyn > 0) alloc((void**)&s->dyn, sizeof(float) * 4 * cfg->n_dyn * (size_t)n);
  alloc((void**)&s->q_sync_dev, sizeof(unsigned) * ((size_t)(n + 127) / 128 + 2));
  // maps are preprocessed in groups whose grids fit a staging budget
  const size_t budget = std::max(max_cells, (size_t)256 << 20);
  uint8_t* staging = nullptr;  // grids, then per-row distances
  PrepMap* mp_dev = nullptr;
  long long* prefix_dev = nullptr;  // [3][n_maps + 1]: words, rows, cells
  alloc((void**)&staging, budget * 2);
  alloc((void**)&mp_dev, sizeof(PrepMap) * n_maps);
  alloc((void**)&prefix_dev, sizeof(long long) * 3 * (n_maps + 1));
  if (e != cudaSuccess) {
    cudaFree(staging);
    cudaFree(mp_dev);
    cudaFree(prefix_dev);
    free_sim(s);
    cuda_fail(e, "cudaMalloc");
    return SG_E_OOM;
  }
  e = cudaMemset(s->clr, 0, (size_t)clr_bytes);  // the zero borders of the skip maps
  std::vector<PrepMap> mp;
  std::vector<long long> pw, pr, pc;
  int m0 = 0;
  while (m0 < n_maps && e == cudaSuccess) {
    mp.clear();
    pw.assign(1, 0);
    pr.assign(1, 0);
    pc.assign(1, 0);
    size_t used = 0;
    int m1 = m0;
    while (m1 < n_maps) {
      const size_t cells = (size_t)map_w[m1] * map_h[m1];
      if (m1 > m0 && used + cells > budget) break;
      PrepMap d;
      d.src = (long long)used;
      d.word_off = md[m1].word_off;
      d.clr_off = md[m1].clr_off;
      d.w = map_w[m1];
      d.h = map_h[m1];
      d.row_words = md[m1].row_words;
      d.clr_ld = md[m1].clr_ld;
      mp.push_back(d);
      e = cudaMemcpyAsync(staging + used, maps_host[m1], cells, cudaMemcpyHostToDevice, 0);
      if (e != cudaSuccess) break;
      used += cells;
      pw.push_back(pw.back() + (long long)d.row_words * d.h);
      pr.push_back(pr.back() + d.h);
      pc.push_back(pc.back() + (long long)cells);
      ++m1;
    }
    if (e != cudaSuccess) break;
    const int nm = m1 - m0;
    e = cudaMemcpyAsync(mp_dev, mp.data(), sizeof(PrepMap) * nm, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(prefix_dev, pw.data(), sizeof(long long) * nm, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(prefix_dev + n_maps + 1, pr.data(), sizeof(long long) * nm, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(prefix_dev + 2 * (n_maps + 1), pc.data(), sizeof(long long) * nm, cudaMemcpyHostToDevice, 0);
    if (e != cudaSuccess) break;
    const long long tw = pw.back(), tr = pr.back(), tc = pc.back();
    k_pack_maps<<<(unsigned)((tw * 32 + 255) / 256), 256>>>(staging, mp_dev, prefix_dev, nm, tw, s->atlas);
    k_clr_rows<<<(unsigned)((tr + 127) / 128), 128>>>(staging, mp_dev, prefix_dev + n_maps + 1, nm, tr,
                                                       staging + budget);
    k_clr_cols<<<(unsigned)((tc + 255) / 256), 256>>>(staging + budget, mp_dev, prefix_dev + 2 * (n_maps + 1), nm,
                                                       tc, s->clr);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();  // the staging buffer is reused by the next group
    m0 = m1;
  }
  cudaFree(staging);
  cudaFree(mp_dev);
  cudaFree(prefix_dev);
  if (e == cudaSuccess) e = cudaMemcpy(s->maps_dev, md.data(), sizeof(MapDesc) * n_maps, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && sec_bytes > 0) e = build_sector_planes(s);
  if (e == cudaSuccess) e = cudaMemcpy(s->env_map_dev, env_map, sizeof(int) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return env_map[a] < env_map[b]; });
    e = cudaMemcpy(s->map_order_dev, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess && env_beams)
    e = cudaMemcpy(s->env_beams_dev, env_beams, sizeof(int) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(s->fstate, 0, sizeof(float) * 9 * (size_t)n);
  if (e == cudaSuccess) e = cudaMemset(s->ustate, 0, sizeof(uint32_t) * 4 * (size_t)n);
  if (e == cudaSuccess) e = cudaMemset(s->status_dev, 0, sizeof(uint32_t));
  if (e == cudaSuccess && s->dyn) e = cudaMemset(s->dyn, 0, sizeof(float) * 4 * cfg->n_dyn * (size_t)n);
  if (e != cudaSuccess) {
    free_sim(s);
    return cuda_fail(e, "sg_sim_create");
  }
  *out = s;
  return SG_OK;
}

extern "C" int sg_sim_destroy(sg_sim_t sim) {
  SG_RANGE("sg_sim_destroy");
  if (!sim) return SG_E_INVAL;
  cudaDeviceSynchronize();
  free_sim(sim);
  return SG_OK;
}

extern "C" int sg_sim_info_get(sg_sim_t sim, sg_sim_info* info) {
  SG_RANGE("sg_sim_info_get");
  if (!sim || !info) return SG_E_INVAL;
  std::memset(info, 0, sizeof(*info));
  info->n_envs = sim->dc.n_envs;
  info->n_beams = sim->dc.B;
  info->obs_dim = sim->dc.obs_dim;
  info->n_maps = sim->n_maps;
  info->atlas_words = sim->atlas_words;
  info->state_bytes = sg_state_bytes(sim);
  info->device = sim->device;
  info->march_sectors = sim->dc.n_sec;
  return SG_OK;
}

long long sg_state_bytes(const sg_sim* s) { return (long long)s->dc.n_envs * (9 * 4 + 4 * 4 + 16 * s->dc.n_dyn); }

extern "C" int sg_sim_reset(sg_sim_t sim, uint64_t seed, float* obs_dev, sg_stream_t stream) {
  SG_RANGE("sg_sim_reset");
  if (!sim) return SG_E_INVAL;
  sim->dc.seed = seed;
  sim->cfg.seed = seed;
  if (sim->dc.n_dyn > 0)
    k_reset<true><<<grid_for(sim->dc.n_envs), 32 * kWarpsPerBlock, 0, stream>>>(sim->dc, sg_sim_ptrs(sim), obs_dev);
  else
    k_reset<false><<<grid_for(sim->dc.n_envs), 32 * kWarpsPerBlock, 0, stream>>>(sim->dc, sg_sim_ptrs(sim), obs_dev);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

extern "C" int sg_sim_step(sg_sim_t sim, const uint8_t* act_dev, float* obs_dev, float* rew_dev,
                           uint8_t* done_dev, float* term_obs_dev, sg_stream_t stream) {
  SG_RANGE("sg_sim_step");
  if (!sim || !act_dev || !obs_dev || !rew_dev || !done_dev) return SG_E_INVAL;
  if (((uintptr_t)obs_dev & 3) || ((uintptr_t)rew_dev & 3) || ((uintptr_t)term_obs_dev & 3)) return SG_E_ALIGN;
  const bool dyn = sim->dc.n_dyn > 0;
  auto kern_for = [dyn](int e) {
    if (e == 6) return dyn ? k_step<true, 6> : k_step<false, 6>;
    if (e == 7) return dyn ? k_step<true, 7> : k_step<false, 7>;
    return dyn ? k_step<true, 8> : k_step<false, 8>;
  };
  const long long n = sim->dc.n_envs;
  if (sim->step_epw == 0) {
    // envs per warp: the count whose grid fills its last wave of resident
    // CTAs best (chosen once per simulator)
    int sms = 0;
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sim->device));
    double best = -1.0;
    for (int e = 8; e >= 6; --e) {
      int bps = 0;
      SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern_for(e), 32 * kStepWarps, 0));
      const long long ctas = (n + kStepWarps * e - 1) / (kStepWarps * e), res = (long long)sms * std::max(bps, 1);
      const double fill = (double)ctas / (double)(((ctas + res - 1) / res) * res);
      if (fill > best + 1e-9) {
        best = fill;
        sim->step_epw = e;
      }
    }
  }
  const int per = kStepWarps * sim->step_epw;
  kern_for(sim->step_epw)<<<(unsigned)((n + per - 1) / per), 32 * kStepWarps, 0, stream>>>(
      sim->dc, sg_sim_ptrs(sim), sim->map_order_dev, act_dev, obs_dev, rew_dev, done_dev, term_obs_dev);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

// Q-network rollouts live with the network (sg_qnet.cu).
int sg_rollout_eps_q(sg_sim* sim, int K, sg_qnet* q, const float* eps, sg_replay* rp, float* obs, float* obs_seq,
                     uint8_t* act_seq, float* rew_seq, uint8_t* done_seq, cudaStream_t stream);

extern "C" int sg_sim_rollout(sg_sim_t sim, int32_t K, int32_t policy, sg_qnet_t qnet, const float* eps_dev,
                              sg_replay_t replay, float* obs_dev, float* obs_seq_dev, uint8_t* act_seq_dev,
                              float* rew_seq_dev, uint8_t* done_seq_dev, sg_stream_t stream) {
  SG_RANGE("sg_sim_rollout");
  if (!sim || K < 1 || K > (1 << 20)) return SG_E_INVAL;
  if (((uintptr_t)obs_dev & 3) || ((uintptr_t)obs_seq_dev & 3) || ((uintptr_t)rew_seq_dev & 3)) return SG_E_ALIGN;
  if (policy == SG_POLICY_RANDOM) {
    if (replay) return SG_E_INVAL;  // transitions are recorded by the Q-policy rollout
    const sg_launch& L = sim->launch;
    const int n = sim->dc.n_envs;
    const SimPtrs sp = sg_sim_ptrs(sim);
    switch (L.kernel) {
      case SG_ROLLOUT_PIPE: {
        const int G = 1 + L.obs_warps;
        const int E = pipe_envs_per_block(L);
        const bool dyn = sim->dc.n_dyn > 0;
        const size_t smem = pipe_smem_bytes(E, dyn);
        const int nblk = (n + E - 1) / E;
        int seg = L.segment < K ? L.segment : 0;  // one segment needs no slicing
        long long grid = nblk;
        if (seg > 0) {
          // items are counted in 32 bits: lengthen the segments if needed
          while ((long long)nblk * ((K + seg - 1) / seg) >= (1ll << 31)) seg *= 2;
          const long long nitems = (long long)nblk * ((K + seg - 1) / seg);
          grid = std::min<long long>(nitems, (long long)sim->persistent_blocks);
          SG_CUDA(cudaMemsetAsync(sim->pipe_sync_dev, 0, sizeof(unsigned) * (size_t)(nblk + 2), stream));
        }
        (dyn ? k_rollout_random_pipe<true> : k_rollout_random_pipe<false>)<<<(unsigned)grid, 32 * G * E, smem,
                                                                          stream>>>(
            sim->dc, sp, K, L.obs_warps, L.order ? sim->map_order_dev : nullptr, seg,
            seg > 0 ? sim->pipe_sync_dev : nullptr, L.wait_iters > 0 ? (unsigned)L.wait_iters : kPipeWaitIters,
            obs_dev, obs_seq_dev, act_seq_dev, rew_seq_dev, done_seq_dev);
        break;
      }
      case SG_ROLLOUT_SPLIT: {
        const int W = L.warps_per_env;
        const int E = L.warps_per_block / W > 0 ? L.warps_per_block / W : 1;
        k_rollout_random_split<<<(n + E - 1) / E, 32 * W * E, 0, stream>>>(
            sim->dc, sp, K, W, obs_dev, obs_seq_dev, act_seq_dev, rew_seq_dev, done_seq_dev);
        break;
      }
      case SG_ROLLOUT_QUEUE: {
        SG_CUDA(cudaMemsetAsync(sim->queue_dev, 0, sizeof(unsigned), stream));
        auto kern = sim->dc.n_dyn > 0 ? k_rollout_random_queue<true> : k_rollout_random_queue<false>;
        kern<<<sim->persistent_blocks, 32 * L.warps_per_block, 0, stream>>>(
            sim->dc, sp, K, L.order ? sim->order_dev : nullptr, sim->queue_dev, obs_dev, obs_seq_dev, act_seq_dev,
            rew_seq_dev, done_seq_dev);
        break;
      }
      default: {
        const int wpb = L.warps_per_block;
        auto kern = sim->dc.n_dyn > 0 ? k_rollout_random<true> : k_rollout_random<false>;
        kern<<<(n + wpb - 1) / wpb, 32 * wpb, 0, stream>>>(sim->dc, sp, K, obs_dev, obs_seq_dev, act_seq_dev,
                                                            rew_seq_dev, done_seq_dev);
      }
    }
    SG_CUDA(cudaGetLastError());
    return SG_OK;
  }
  if (policy == SG_POLICY_EPS_Q) {
    if (!qnet || !eps_dev) return SG_E_INVAL;
    return sg_rollout_eps_q(sim, K, qnet, eps_dev, replay, obs_dev, obs_seq_dev, act_seq_dev, rew_seq_dev,
                            done_seq_dev, stream);
  }
  return SG_E_INVAL;
}

extern "C" int sg_sim_set_launch(sg_sim_t sim, const sg_launch* cfg) {
  SG_RANGE("sg_sim_set_launch");
  if (!sim || !cfg) return SG_E_INVAL;
  const sg_launch L = *cfg;
  auto pow2 = [](int v) { return v == 1 || v == 2 || v == 4 || v == 8 || v == 16; };
  switch (L.kernel) {
    case SG_ROLLOUT_GRID:
      if (!pow2(L.warps_per_block)) return SG_E_INVAL;
      break;
    case SG_ROLLOUT_QUEUE:
      if (!pow2(L.warps_per_block) || L.blocks_per_sm < 0 || L.blocks_per_sm > 64 || L.order < 0 || L.order > 1)
        return SG_E_INVAL;
      break;
    case SG_ROLLOUT_SPLIT:
      // the kernel is compiled for at most 256 threads per CTA; its warps
      // replay the pose chain without the discs
      if (sim->dc.n_dyn > 0) return SG_E_INVAL;
      if (L.warps_per_env < 1 || L.warps_per_env > 8 || L.warps_per_block < 1 || L.warps_per_block > 8)
        return SG_E_INVAL;
      break;
    case SG_ROLLOUT_PIPE:
      if (L.obs_warps < 1 || L.obs_warps > 15 || L.warps_per_block < 1 || L.warps_per_block > 16 || L.order < 0 ||
          L.order > 1)
        return SG_E_INVAL;
      if (L.segment < 0 || L.segment > (1 << 20) || L.segment % kPipeChunk != 0 || L.wait_iters < 0)
        return SG_E_INVAL;
      break;
    default:
      return SG_E_INVAL;
  }
  int sms = 0;
  SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sim->device));
  int bps = L.blocks_per_sm;
  if (L.kernel == SG_ROLLOUT_PIPE) {
    const int E = pipe_envs_per_block(L);
    const bool dyn = sim->dc.n_dyn > 0;
    const size_t smem = pipe_smem_bytes(E, dyn);
    auto kern = dyn ? k_rollout_random_pipe<true> : k_rollout_random_pipe<false>;
    SG_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (L.segment > 0) {
      // time slicing: a resident grid and the per-CTA segment flags
      SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern,
                                                            32 * (1 + L.obs_warps) * E, smem));
      if (bps < 1) bps = 1;
      if (L.blocks_per_sm > 0) bps = std::min(bps, L.blocks_per_sm);
      const size_t words = (size_t)((sim->dc.n_envs + E - 1) / E) + 2;
      if (words > sim->pipe_sync_words) {
        cudaFree(sim->pipe_sync_dev);
        sim->pipe_sync_dev = nullptr;
        sim->pipe_sync_words = 0;
        SG_CUDA(cudaMalloc(&sim->pipe_sync_dev, sizeof(unsigned) * words));
        sim->pipe_sync_words = words;
      }
    }
  }
  if (L.kernel == SG_ROLLOUT_QUEUE && bps == 0) {
    SG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &bps, sim->dc.n_dyn > 0 ? k_rollout_random_queue<true> : k_rollout_random_queue<false>,
        32 * L.warps_per_block, 0));
    if (bps < 1) bps = 1;
  }
  if (L.kernel == SG_ROLLOUT_QUEUE && L.order == 1 && !sim->order_dev) {
    // longest first: beams x map size, ties by env index
    const int n = sim->dc.n_envs;
    std::vector<int> beams((size_t)n, sim->dc.B), emap((size_t)n);
    SG_CUDA(cudaMemcpy(emap.data(), sim->env_map_dev, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (sim->env_beams_dev) SG_CUDA(cudaMemcpy(beams.data(), sim->env_beams_dev, sizeof(int) * n, cudaMemcpyDeviceToHost));
    std::vector<int> order((size_t)n);
    std::vector<double> cost((size_t)n);
    for (int i = 0; i < n; ++i) {
      order[i] = i;
      const sg::MapDesc& m = sim->maps_host[emap[i]];
      cost[i] = env_cost(beams[i], m.w, m.h);
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    SG_CUDA(cudaMalloc(&sim->order_dev, sizeof(int) * n));
    SG_CUDA(cudaMemcpy(sim->order_dev, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  }
  if (L.kernel == SG_ROLLOUT_QUEUE && !sim->queue_dev) SG_CUDA(cudaMalloc(&sim->queue_dev, sizeof(unsigned)));
  sim->launch = L;
  sim->persistent_blocks =
      (L.kernel == SG_ROLLOUT_QUEUE || (L.kernel == SG_ROLLOUT_PIPE && L.segment > 0)) ? bps * sms : 0;
  return SG_OK;
}

extern "C" int sg_sim_get_launch(sg_sim_t sim, sg_launch* cfg) {
  SG_RANGE("sg_sim_get_launch");
  if (!sim || !cfg) return SG_E_INVAL;
  *cfg = sim->launch;
  return SG_OK;
}

extern "C" int sg_sim_get_state(sg_sim_t sim, void* host_buf, size_t* bytes) {
  SG_RANGE("sg_sim_get_state");
  if (!sim || !bytes) return SG_E_INVAL;
  const size_t need = (size_t)sg_state_bytes(sim);
  if (!host_buf) {
    *bytes = need;
    return SG_OK;
  }
  if (*bytes < need) return SG_E_INVAL;
  const size_t n = (size_t)sim->dc.n_envs;
  SG_CUDA(cudaDeviceSynchronize());
  SG_CUDA(cudaMemcpy(host_buf, sim->fstate, 9 * 4 * n, cudaMemcpyDeviceToHost));
  SG_CUDA(cudaMemcpy((char*)host_buf + 9 * 4 * n, sim->ustate, 4 * 4 * n, cudaMemcpyDeviceToHost));
  if (sim->dc.n_dyn > 0)
    SG_CUDA(cudaMemcpy((char*)host_buf + 13 * 4 * n, sim->dyn, 16 * (size_t)sim->dc.n_dyn * n, cudaMemcpyDeviceToHost));
  *bytes = need;
  return SG_OK;
}

extern "C" int sg_sim_set_state(sg_sim_t sim, const void* host_buf, size_t bytes) {
  SG_RANGE("sg_sim_set_state");
  if (!sim || !host_buf) return SG_E_INVAL;
  const size_t need = (size_t)sg_state_bytes(sim);
  if (bytes != need) return SG_E_INVAL;
  const size_t n = (size_t)sim->dc.n_envs;
  SG_CUDA(cudaDeviceSynchronize());
  SG_CUDA(cudaMemcpy(sim->fstate, host_buf, 9 * 4 * n, cudaMemcpyHostToDevice));
  SG_CUDA(cudaMemcpy(sim->ustate, (const char*)host_buf + 9 * 4 * n, 4 * 4 * n, cudaMemcpyHostToDevice));
  if (sim->dc.n_dyn > 0)
    SG_CUDA(cudaMemcpy(sim->dyn, (const char*)host_buf + 13 * 4 * n, 16 * (size_t)sim->dc.n_dyn * n,
                       cudaMemcpyHostToDevice));
  return SG_OK;
}

extern "C" int sg_sim_set_state_async(sg_sim_t sim, const void* host_buf, size_t bytes, sg_stream_t stream) {
  SG_RANGE("sg_sim_set_state_async");
  if (!sim || !host_buf) return SG_E_INVAL;
  const size_t need = (size_t)sg_state_bytes(sim);
  if (bytes != need) return SG_E_INVAL;
  const size_t n = (size_t)sim->dc.n_envs;
  const cudaStream_t st = (cudaStream_t)stream;
  SG_CUDA(cudaMemcpyAsync(sim->fstate, host_buf, 9 * 4 * n, cudaMemcpyHostToDevice, st));
  SG_CUDA(cudaMemcpyAsync(sim->ustate, (const char*)host_buf + 9 * 4 * n, 4 * 4 * n, cudaMemcpyHostToDevice, st));
  if (sim->dc.n_dyn > 0)
    SG_CUDA(cudaMemcpyAsync(sim->dyn, (const char*)host_buf + 13 * 4 * n, 16 * (size_t)sim->dc.n_dyn * n,
                            cudaMemcpyHostToDevice, st));
  return SG_OK;
}

extern "C" int sg_sim_get_atlas(sg_sim_t sim, uint32_t* atlas_host, size_t* words, int64_t* offs_host,
                                int32_t* row_words_host) {
  SG_RANGE("sg_sim_get_atlas");
  if (!sim) return SG_E_INVAL;
  if (atlas_host) {
    if (!words || *words < (size_t)sim->atlas_words) return SG_E_INVAL;
    SG_CUDA(cudaDeviceSynchronize());
    SG_CUDA(cudaMemcpy(atlas_host, sim->atlas, (size_t)sim->atlas_words * 4, cudaMemcpyDeviceToHost));
  }
  if (words) *words = (size_t)sim->atlas_words;
  for (int m = 0; m < sim->n_maps; ++m) {
    if (offs_host) offs_host[m] = sim->maps_host[m].word_off;
    if (row_words_host) row_words_host[m] = sim->maps_host[m].row_words;
  }
  return SG_OK;
}

extern "C" int sg_sim_get_clearance(sg_sim_t sim, uint8_t* host, size_t* bytes, int64_t* offs_host) {
  SG_RANGE("sg_sim_get_clearance");
  if (!sim || !bytes) return SG_E_INVAL;
  size_t total = 0;
  for (int m = 0; m < sim->n_maps; ++m) total += (size_t)sim->maps_host[m].w * sim->maps_host[m].h;
  if (host) {
    if (*bytes < total) return SG_E_INVAL;
    SG_CUDA(cudaDeviceSynchronize());
    size_t off = 0;
    for (int m = 0; m < sim->n_maps; ++m) {
      const MapDesc& d = sim->maps_host[m];
      SG_CUDA(cudaMemcpy2D(host + off, (size_t)d.w, sim->clr + d.clr_off, (size_t)d.clr_ld, (size_t)d.w,
                           (size_t)d.h, cudaMemcpyDeviceToHost));
      off += (size_t)d.w * d.h;
    }
  }
  *bytes = total;
  if (offs_host) {
    int64_t off = 0;
    for (int m = 0; m < sim->n_maps; ++m) {
      offs_host[m] = off;
      off += (int64_t)sim->maps_host[m].w * sim->maps_host[m].h;
    }
  }
  return SG_OK;
}

extern "C" int sg_sim_get_sector_skip(sg_sim_t sim, uint8_t* host, size_t* bytes, int64_t* offs_host) {
  SG_RANGE("sg_sim_get_sector_skip");
  if (!sim || !bytes) return SG_E_INVAL;
  const int S = sim->dc.n_sec > 1 ? sim->dc.n_sec : 0;
  size_t total = 0;
  for (int m = 0; m < sim->n_maps; ++m) total += (size_t)S * sim->maps_host[m].w * sim->maps_host[m].h;
  if (host && total > 0) {
    if (*bytes < total) return SG_E_INVAL;
    SG_CUDA(cudaDeviceSynchronize());
    size_t off = 0;
    for (int m = 0; m < sim->n_maps; ++m) {
      const MapDesc& d = sim->maps_host[m];
      for (int p = 0; p < S; ++p) {
        SG_CUDA(cudaMemcpy2D(host + off, (size_t)d.w, sim->sec + d.sec_off + (long long)p * d.sec_plane,
                             (size_t)d.clr_ld, (size_t)d.w, (size_t)d.h, cudaMemcpyDeviceToHost));
        off += (size_t)d.w * d.h;
      }
    }
  }
  *bytes = total;
  if (offs_host) {
    int64_t off = 0;
    for (int m = 0; m < sim->n_maps; ++m) {
      offs_host[m] = off;
      off += (int64_t)S * sim->maps_host[m].w * sim->maps_host[m].h;
    }
  }
  return SG_OK;
}

#ifdef SG_DEBUG_BOUNDS
int sg_take_debug_bounds_qnet(unsigned* v);  // sg_qnet.cu
#endif

extern "C" int sg_sim_status(sg_sim_t sim, uint32_t* device_status) {
  SG_RANGE("sg_sim_status");
  if (!sim || !device_status) return SG_E_INVAL;
  uint32_t v = 0;
  SG_CUDA(cudaDeviceSynchronize());
  SG_CUDA(cudaMemcpy(&v, sim->status_dev, 4, cudaMemcpyDeviceToHost));
  SG_CUDA(cudaMemset(sim->status_dev, 0, 4));
#ifdef SG_DEBUG_BOUNDS
  unsigned b = 0, bq = 0, z = 0;
  SG_CUDA(cudaMemcpyFromSymbol(&b, g_debug_bounds, sizeof(unsigned)));
  SG_CUDA(cudaMemcpyToSymbol(g_debug_bounds, &z, sizeof(unsigned)));
  if (int rc = sg_take_debug_bounds_qnet(&bq)) return rc;
  if (b | bq) v |= SG_DEV_BOUNDS;
#endif
  *device_status = v;
  return v ? SG_E_DEVICE : SG_OK;
}

extern "C" const char* sg_strerror(int code) {
  switch (code) {
    case SG_OK: return "ok";
    case SG_E_INVAL: return "invalid argument";
    case SG_E_ALIGN: return "misaligned pointer";
    case SG_E_OOM: return "out of memory";
    case SG_E_CUDA: return "CUDA runtime error";
    case SG_E_DEVICE: return "device reported an error";
    case SG_E_TIMEOUT: return "device wait timed out";
    default: return "unknown error";
  }
}

extern "C" const char* sg_last_cuda_error(void) { return g_cuda_err; }
