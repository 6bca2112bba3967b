// sg_device.cuh -- device-side building blocks of the vectorized Sparrow step
// (paper arxiv 2305.04180, Sec. 3.2).  One warp simulates one environment:
// the scalar part of the step (kinematics, reward, reset draws) runs
// redundantly in every lane, so that no shuffle is needed to share it, while
// the LiDAR beams, the collision disc rows and the observation stores are
// spread over the lanes.
//
// Floating point: this file is compiled with -fmad=false, so every a*b+c is a
// rounded multiply followed by a rounded add; fmaf() appears exactly where the
// step definition fuses.  Divisions and square roots are IEEE (no fast math).
// Under these rules the step is a fixed float32 expression tree, and its
// discrete decisions (hit index, collision, arrival, reset) are reproducible
// bit for bit by any IEEE float32 evaluation of the same tree.
#pragma once

#include <cstdint>

namespace sg {

constexpr unsigned kFull = 0xffffffffu;

// Debug build (SG_DEBUG_BOUNDS): SG_IN_BOUNDS(cond) is cond, and a false
// cond latches a per-translation-unit device flag that sg_sim_status reports
// as SG_DEV_BOUNDS; the caller then skips the access.  Regular build: true.
#ifdef SG_DEBUG_BOUNDS
static __device__ unsigned g_debug_bounds;
__device__ __forceinline__ bool sg_in_bounds(bool ok) {
  if (!ok) atomicOr(&g_debug_bounds, 1u);
  return ok;
}
#define SG_IN_BOUNDS(cond) sg_in_bounds(cond)
#else
#define SG_IN_BOUNDS(cond) true
#endif
constexpr uint32_t kStreamReset = 1;
constexpr uint32_t kStreamNoise = 2;
constexpr uint32_t kStreamAction = 3;
constexpr uint32_t kNoAction = 255;
constexpr float kPi = 3.14159265358979323846f;
constexpr float kTwoPow24Inv = 5.9604644775390625e-08f;

// Atlas entry of one map.  Bits: row cy starts at word_off + cy * row_words.
// Clearance: byte clr_off + cy * w + cx holds min(255, Chebyshev distance in
// cells from (cx, cy) to the nearest occupied cell, cells outside the map
// counting as occupied); 0 exactly on occupied cells.
// Skip maps (the march's acceleration structure) carry a border of
// kClrBorder zero cells on every side, so a march that starts inside the map
// needs no bounds test (see march()).
constexpr int kClrBorder = 2;

struct MapDesc {
  long long word_off;
  long long clr_off;   // interior cell (0, 0) of the map's skip map
  long long sec_off;   // interior cell (0, 0) of sector plane 0 (see sector skip maps below)
  long long sec_plane; // bytes between consecutive sector planes of the map
  int w, h;
  int row_words;
  int clr_ld;          // row stride of the skip map and of the sector planes, w + 2 * kClrBorder
};

// Sector skip maps (optional, n_sec > 1 planes per map; an acceleration
// structure of the march, not part of the step's definition).  The
// directions of travel are cut into n_sec equal sectors; sector s holds the
// directions whose angle lies in [-pi + s 2pi/n_sec, -pi + (s+1) 2pi/n_sec).
// Plane s stores, for every free cell c, a number J >= 1 of march samples
// that can be skipped by a ray of a sector-s direction whose current sample
// lies in c: J = max(ceil(SC - 0.01), Chebyshev skip of c), where SC is the
// smallest distance from a point of c, along a direction of the sector
// widened by 0.01 rad on each side, to a point of an occupied or outside
// cell, capped at kSecRadius.  The planes have the skip map's layout (zero
// border, 0 on occupied cells).  Why J is exact for march steps <= 1 cell:
// from sample k (in c) the displacement to sample k + j is j u plus two
// float32 roundings (< 0.003 cells on maps up to 16384), so it points
// within 0.003 rad of u for j >= 1 and is shorter than j + 0.003 < SC for
// j < J; the samples k+1 .. k+J-1 therefore lie in free cells and the first
// sample that can hit is k + J, as with the Chebyshev skip.
constexpr int kSecRadius = 48;
constexpr int kMaxSectors = 32;

// Launch-time copy of the configuration (float32 values).
struct DevCfg {
  int n_envs, B, obs_dim, n_actions, t_max, kmax, delay_lo, delay_span;
  int skip_ok;      // march_step <= 1: clearance skipping is exact
  int clr_collide;  // skip value from which the collision disc cannot touch a wall
  int n_sec;        // sector skip planes per map (1: the Chebyshev skip map only)
  float sec_scale;  // n_sec / (2 pi): beam angle beta -> sector of u = -(cos beta, sin beta)
  float fov, half_fov, range_max, delta, robot_r, goal_r, near_dist, start_offset, jitter;
  float dt_lo, dt_hi, k_lo, k_hi, cap_lo, cap_hi, sig_lo, sig_hi;
  float v_nom, w_nom;
  float av[8], aw[8];
  unsigned long long seed;
  // dynamic obstacles (n_dyn = 0: none)
  int n_dyn;
  float dyn_r, dyn_r2;  // disc radius r_o and r_o^2
  float dyn_rr2;        // (robot_r + r_o)^2
  float dyn_keep2;      // squared keep-out distance from S and G at the draws
  float dyn_vlo, dyn_vhi;
  float dyn_re;         // radius of the scan's candidate band, r_o + delta + 0.25
};

// Device buffers of a simulator (structure of arrays, stride n).
struct SimPtrs {
  float* f;               // [9][n]: x y phi vl va dt K cap sigma
  uint32_t* u;            // [4][n]: ep_step ep_id t fifo
  const uint32_t* atlas;  // bit-packed maps
  const uint8_t* clr;     // skip maps (see march())
  const uint8_t* sec;     // sector skip planes (n_sec > 1), else null
  const MapDesc* maps;
  const int* env_map;
  const int* env_beams;   // nullptr: every env uses B beams
  uint32_t* status;       // SG_DEV_* bits
  float* dyn;             // [4 n_dyn][n]: obstacle o at rows 4o..4o+3 (x y vx vy); null when n_dyn = 0
  int n;
  int pad;
};

// Registers of one environment.
struct Env {
  float x, y, phi, vl, va, dt, K, cap, sigma;
  uint32_t ep_step, ep_id, t, fifo;  // fifo: q0 | q1 << 8 | delay << 16
  float sphi, cphi;                  // f_sincos(phi), kept with phi (not stored)
};

// ------------------------------------------------------------- RNG
// SplitMix64 (Steele, Lea & Flood 2014): value of the generator seeded with s
// after c+1 steps; nesting it hashes several counters.
__device__ __forceinline__ uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm_at(uint64_t s, uint64_t c) {
  return sm_mix(s + (c + 1ull) * 0x9E3779B97F4A7C15ull);
}
__device__ __forceinline__ float u24_hi(uint64_t h) {
  return (float)(uint32_t)(h >> 40) * kTwoPow24Inv;
}
__device__ __forceinline__ float u24_mid(uint64_t h) {
  return (float)(uint32_t)((h >> 16) & 0xFFFFFFu) * kTwoPow24Inv;
}

// ------------------------------------------------- float32 functions
// sin and cos together: Cody-Waite reduction by the nearest multiple of
// pi/2 (two-word pi/2 through fma), Taylor polynomials of sin (degree 11)
// and cos (degree 12) in Horner form, quadrant from q mod 4.
__device__ __forceinline__ void f_sincos(float a, float& s, float& c) {
  const float q = rintf(a * 0.636619772f);
  const int qi = (int)q;
  float r = fmaf(-q, 1.57079637050628662109375f, a);
  r = fmaf(-q, -4.371139000186243e-08f, r);
  const float z = r * r;
  float ps = fmaf(z, -2.505210838544172e-08f, 2.7557319223985893e-06f);
  ps = fmaf(z, ps, -1.984126984126984e-04f);
  ps = fmaf(z, ps, 8.333333333333333e-03f);
  ps = fmaf(z, ps, -1.6666666666666666e-01f);
  const float sr = fmaf(r * z, ps, r);
  float pc = fmaf(z, 2.08767569878681e-09f, -2.755731922398589e-07f);
  pc = fmaf(z, pc, 2.48015873015873e-05f);
  pc = fmaf(z, pc, -1.388888888888889e-03f);
  pc = fmaf(z, pc, 4.1666666666666664e-02f);
  pc = fmaf(z, pc, -0.5f);
  const float cr = fmaf(z, pc, 1.0f);
  switch (qi & 3) {
    case 0: s = sr; c = cr; break;
    case 1: s = cr; c = -sr; break;
    case 2: s = -sr; c = -cr; break;
    default: s = -cr; c = sr; break;
  }
}

// atan2 by octant reduction, the identity atan t = pi/4 + atan((t-1)/(t+1))
// above tan(pi/8), and the alternating series of atan to degree 21.
// Coefficients are the floats nearest 1/n.
__device__ __forceinline__ float f_atan2(float y, float x) {
  const float ax = fabsf(x), ay = fabsf(y);
  if (ax == 0.0f && ay == 0.0f) return 0.0f;
  const bool swap = ay > ax;
  const float num = swap ? ax : ay;
  const float den = swap ? ay : ax;
  float t = num / den;
  float base = 0.0f;
  if (t > 0.414213562373095f) {
    t = (t - 1.0f) / (t + 1.0f);
    base = 0.785398163397448f;
  }
  const float w = t * t;
  float p = fmaf(w, 0.04761905f, -0.05263158f);
  p = fmaf(w, p, 0.05882353f);
  p = fmaf(w, p, -0.06666667f);
  p = fmaf(w, p, 0.07692308f);
  p = fmaf(w, p, -0.09090909f);
  p = fmaf(w, p, 0.11111111f);
  p = fmaf(w, p, -0.14285715f);
  p = fmaf(w, p, 0.2f);
  p = fmaf(w, p, -0.33333334f);
  p = fmaf(w, p, 1.0f);
  float a = base + t * p;
  if (swap) a = 1.57079632679490f - a;
  if (x < 0.0f) a = 3.14159265358979f - a;
  if (y < 0.0f) a = -a;
  return a;
}

// Natural log of a positive normal float: x = m 2^e with m in
// (sqrt(1/2), sqrt(2)], ln m = 2 atanh((m-1)/(m+1)) by its odd series to
// degree 13, plus e ln 2 split in two words.
__device__ __forceinline__ float f_log(float x) {
  const uint32_t bits = __float_as_uint(x);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > 1.41421356237310f) {
    m = m * 0.5f;
    e = e + 1;
  }
  const float z = (m - 1.0f) / (m + 1.0f);
  const float w = z * z;
  float p = fmaf(w, 0.07692308f, 0.09090909f);
  p = fmaf(w, p, 0.11111111f);
  p = fmaf(w, p, 0.14285715f);
  p = fmaf(w, p, 0.2f);
  p = fmaf(w, p, 0.33333334f);
  p = fmaf(w, p, 1.0f);
  const float t = z * p;
  const float lnm = t + t;
  const float ef = (float)e;
  const float lo = fmaf(ef, 1.4286068203094172e-06f, lnm);
  return fmaf(ef, 0.693145751953125f, lo);
}

// ------------------------------------------------------- state I/O
__device__ __forceinline__ Env load_env(const SimPtrs& p, int i) {
  Env s;
  const int n = p.n;
  s.x = p.f[0 * n + i];
  s.y = p.f[1 * n + i];
  s.phi = p.f[2 * n + i];
  s.vl = p.f[3 * n + i];
  s.va = p.f[4 * n + i];
  s.dt = p.f[5 * n + i];
  s.K = p.f[6 * n + i];
  s.cap = p.f[7 * n + i];
  s.sigma = p.f[8 * n + i];
  s.ep_step = p.u[0 * n + i];
  s.ep_id = p.u[1 * n + i];
  s.t = p.u[2 * n + i];
  s.fifo = p.u[3 * n + i];
  f_sincos(s.phi, s.sphi, s.cphi);
  return s;
}

__device__ __forceinline__ void store_env(const SimPtrs& p, int i, const Env& s) {
  const int n = p.n;
  p.f[0 * n + i] = s.x;
  p.f[1 * n + i] = s.y;
  p.f[2 * n + i] = s.phi;
  p.f[3 * n + i] = s.vl;
  p.f[4 * n + i] = s.va;
  p.f[5 * n + i] = s.dt;
  p.f[6 * n + i] = s.K;
  p.f[7 * n + i] = s.cap;
  p.f[8 * n + i] = s.sigma;
  p.u[0 * n + i] = s.ep_step;
  p.u[1 * n + i] = s.ep_id;
  p.u[2 * n + i] = s.t;
  p.u[3 * n + i] = s.fifo;
}

// -------------------------------------------------------- geometry
struct Layout {
  float sx, sy, gx, gy, D;
};

// Start S (lower left), goal G (upper right) and planning distance D = |G-S|.
__device__ __forceinline__ Layout layout_of(const DevCfg& c, const MapDesc& m) {
  Layout L;
  L.sx = c.start_offset;
  L.sy = c.start_offset;
  L.gx = (float)m.w - c.start_offset;
  L.gy = (float)m.h - c.start_offset;
  const float ex = L.gx - L.sx, ey = L.gy - L.sy;
  L.D = sqrtf(fmaf(ex, ex, ey * ey));
  return L;
}

// Fixed-step ray march: sample k = 1..kmax at (fma(k d, ux, x), fma(k d, uy, y));
// the first sample whose cell is occupied or outside the map is the hit.
//
// The march reads the skip map instead of the bits: with c the clearance of a
// cell (0 on occupied cells; c >= 1 says every cell within Chebyshev distance
// c - 1 is free and inside the map), the map holds s = 0 for c = 0 and
// s = max(1, c - 1) otherwise, and a border of kClrBorder zero cells around
// the map.  With march_step <= 1 and |ux|, |uy| <= 1 the sample cell moves by
// at most j + 1 cells per axis over j samples (j cells of travel plus one for
// the rounding of the two fma results, which is below 2^-9 cells for maps up
// to 16384 cells), so the samples k+1 .. k+c-2 all lie in free cells and the
// next sample that can hit is k + s: the hit index is the same as testing
// every sample.  The same bound puts the next sample at most c cells from the
// current one (2 when c = 1), so from an origin inside the map no sample
// leaves the border before a zero stops the march: that loop has no bounds
// test.  Origins outside the map, and steps above one cell (no skipping), use
// the bounds-tested loop.  The same loop runs on a sector plane (see
// MapDesc): its values are skips of the same meaning for the rays of its
// sector, with the same zero border.
// Conversions on the FP32 and integer pipes instead of the conversion unit:
// for an integer or float v with |v| < 2^22, v + 1.5 * 2^23 lies in
// [2^23, 2^24), where the floats are exactly the integers, so the bit pattern
// of that sum minus the pattern of 1.5 * 2^23 is the integer.  (uint)k +
// pattern, reinterpreted, minus 1.5 * 2^23 is (float)k; the sum rounded down
// is floor(v).  Sample cells lie in [-2, 16386), the map offset iy * ld + ix
// in int range, so it is taken modulo 2^32 from the two patterns (bias
// folds in the two subtracted patterns).
constexpr float kMarchMagic = 12582912.0f;
constexpr uint32_t kMarchMagicBits = 0x4B400000u;

// Whether a march from (x, y) takes the unbounded skipping loop.
template <bool kUnitStep>
__device__ __forceinline__ bool march_fast(int W, int H, float x, float y, int skip_ok) {
  return (kUnitStep || skip_ok) && x >= 0.0f && y >= 0.0f && x < (float)W && y < (float)H;
}

// Skip value at sample k of the unbounded loop (0 = a hit there).
template <bool kUnitStep>
__device__ __forceinline__ int march_skip_at(const uint8_t* __restrict__ clr, int W, int H, int ld, uint32_t bias,
                                             float x, float y, float ux, float uy, float delta, int k) {
  const float kf = __uint_as_float((uint32_t)k + kMarchMagicBits) - kMarchMagic;
  // with a unit step, (float)k * 1.0f is (float)k exactly
  const float t = kUnitStep ? kf : kf * delta;
  const uint32_t bx = __float_as_uint(__fadd_rd(fmaf(t, ux, x), kMarchMagic));
  const uint32_t by = __float_as_uint(__fadd_rd(fmaf(t, uy, y), kMarchMagic));
  // the sample cell (ix, iy) = (bx, by) - pattern(1.5 * 2^23), inside the border
  if (!SG_IN_BOUNDS((int)(bx - kMarchMagicBits) >= -kClrBorder && (int)(by - kMarchMagicBits) >= -kClrBorder &&
                    (int)(bx - kMarchMagicBits) < W + kClrBorder && (int)(by - kMarchMagicBits) < H + kClrBorder))
    return 0;
  return __ldg(clr + (int)(by * (uint32_t)ld + bx + bias));
}
__device__ __forceinline__ uint32_t march_bias(int ld) { return 0u - kMarchMagicBits * (uint32_t)(ld + 1); }

// s1 >= 0: the caller checked march_fast and loaded sample 1's skip value
// (march_skip_at, k = 1) ahead, so that its latency overlapped other work.
template <bool kUnitStep>
__device__ __forceinline__ int march(const uint8_t* __restrict__ clr, int W, int H, int ld, float x, float y,
                                     float ux, float uy, float delta, int kmax, int skip_ok, int s1 = -1) {
  int k = 1;
  if (s1 >= 0 || march_fast<kUnitStep>(W, H, x, y, skip_ok)) {
    const uint32_t bias = march_bias(ld);
    int s = s1 >= 0 ? s1 : march_skip_at<kUnitStep>(clr, W, H, ld, bias, x, y, ux, uy, delta, k);
    for (;;) {
      if (s == 0) return k;
      k += s;
      if (k > kmax) return kmax + 1;
      s = march_skip_at<kUnitStep>(clr, W, H, ld, bias, x, y, ux, uy, delta, k);
    }
  }
  while (k <= kmax) {
    const float t = kUnitStep ? (float)k : (float)k * delta;
    const float px = fmaf(t, ux, x);
    const float py = fmaf(t, uy, y);
    const int ix = __float2int_rd(px), iy = __float2int_rd(py);
    if ((unsigned)ix >= (unsigned)W || (unsigned)iy >= (unsigned)H) return k;
    const int s = __ldg(clr + iy * ld + ix);
    if (s == 0) return k;
    k += (kUnitStep || skip_ok) ? s : 1;
  }
  return kmax + 1;
}

// Robot disc against the occupied cells: the centre leaving the map, or an
// occupied cell centre within robot_r (fma(dx,dx,dy*dy) <= r*r).  This part
// tests the bit rows of the candidate box around an in-map centre: lanes take
// rows, only set bits reach the distance test.
__device__ __forceinline__ bool collide_rows_warp(const DevCfg& c, const MapDesc& m,
                                                  const uint32_t* __restrict__ rows, float x, float y, int lane) {
  const float r = c.robot_r;
  const float r2 = r * r;
  int cx0 = (int)floorf(x - r) - 1, cx1 = (int)floorf(x + r) + 1;
  int cy0 = (int)floorf(y - r) - 1, cy1 = (int)floorf(y + r) + 1;
  cx0 = max(cx0, 0);
  cy0 = max(cy0, 0);
  cx1 = min(cx1, m.w - 1);
  cy1 = min(cy1, m.h - 1);
  bool hit = false;
  for (int cy = cy0 + lane; cy <= cy1; cy += 32) {
    const uint32_t* row = rows + (long long)cy * m.row_words;
    for (int wd = cx0 >> 5; wd <= (cx1 >> 5); ++wd) {
      const int lo = max(cx0 - wd * 32, 0), hi = min(cx1 - wd * 32, 31);
      const uint32_t mask = (0xFFFFFFFFu >> (31 - hi)) & (0xFFFFFFFFu << lo);
      if (!SG_IN_BOUNDS(cy >= 0 && cy < m.h && wd >= 0 && wd < m.row_words)) continue;
      uint32_t bits = __ldg(row + wd) & mask;
      while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1;
        const float dx = ((float)(wd * 32 + b) + 0.5f) - x;
        const float dy = ((float)cy + 0.5f) - y;
        if (fmaf(dx, dx, dy * dy) <= r2) hit = true;
      }
    }
  }
  return __any_sync(kFull, hit);
}

// The whole test.  Every occupied cell centre is at least clearance - 0.5
// cells away from a point of the centre's cell, so a large enough clearance
// there (skip value >= clr_collide, i.e. clearance >= ceil(r) + 2) rules out
// any occupied cell within robot_r without reading the rows.
__device__ __forceinline__ bool collide_warp(const DevCfg& c, const MapDesc& m, const uint32_t* __restrict__ rows,
                                             const uint8_t* __restrict__ clr, float x, float y, int lane) {
  if (x < 0.0f || y < 0.0f || x >= (float)m.w || y >= (float)m.h) return true;
  const int own = __ldg(clr + __float2int_rd(y) * m.clr_ld + __float2int_rd(x));
  if (own >= c.clr_collide) return false;
  return collide_rows_warp(c, m, rows, x, y, lane);
}

// ------------------------------------------------ dynamic obstacles
// Optional moving discs (the extension Sec. 5 names as the simulator's next
// capability).  Each env has n_dyn discs of radius r_o moving in straight
// lines: per step, after the robot's motion, a disc advances by dt * v (the
// env's control interval); a centre leaving [r_o, W - r_o] (resp. H) is
// mirrored back and that velocity component flips; a centre that would enter
// an occupied cell stays put and the velocity reverses.  The robot collides
// with a disc when the centres are within robot_r + r_o, and a LiDAR sample
// inside a disc is a hit.  Discs are re-drawn at every episode start.
constexpr int kMaxDyn = 8;

struct Obst {
  float x, y, vx, vy;
};
// Disc centres of one env, the same in every lane of the warp (or in shared
// memory for the lane-per-env step).
struct Discs {
  float x[kMaxDyn], y[kMaxDyn];
};

__device__ __forceinline__ Obst load_obst(const SimPtrs& p, int o, int i) {
  const int n = p.n;
  Obst b;
  b.x = p.dyn[(4 * o + 0) * n + i];
  b.y = p.dyn[(4 * o + 1) * n + i];
  b.vx = p.dyn[(4 * o + 2) * n + i];
  b.vy = p.dyn[(4 * o + 3) * n + i];
  return b;
}

__device__ __forceinline__ void store_obst(const SimPtrs& p, int o, int i, const Obst& b) {
  const int n = p.n;
  p.dyn[(4 * o + 0) * n + i] = b.x;
  p.dyn[(4 * o + 1) * n + i] = b.y;
  p.dyn[(4 * o + 2) * n + i] = b.vx;
  p.dyn[(4 * o + 3) * n + i] = b.vy;
}

// Mirror coordinate v into [lo, hi]; flips vel when it mirrors.
__device__ __forceinline__ float dyn_reflect(float v, float lo, float hi, float& vel) {
  if (v < lo) {
    v = lo + (lo - v);
    vel = -vel;
  } else if (v > hi) {
    v = hi - (v - hi);
    vel = -vel;
  }
  return fminf(fmaxf(v, lo), hi);
}

// One motion step of a disc of map m (skip map clr: 0 exactly on occupied
// cells) with control interval dt.
__device__ __forceinline__ void dyn_move(const DevCfg& c, const MapDesc& m, const uint8_t* __restrict__ clr, float dt,
                                         Obst& b) {
  const float r = c.dyn_r;
  const float hx = (float)m.w - r, hy = (float)m.h - r;
  float vx = b.vx, vy = b.vy;
  float nx = b.x + dt * vx;
  float ny = b.y + dt * vy;
  nx = dyn_reflect(nx, r, hx, vx);
  ny = dyn_reflect(ny, r, hy, vy);
  // nx in [r, W - r] with r > 0: the cell is inside the map
  if (__ldg(clr + __float2int_rd(ny) * m.clr_ld + __float2int_rd(nx)) == 0) {
    b.vx = -b.vx;
    b.vy = -b.vy;
    return;
  }
  b.x = nx;
  b.y = ny;
  b.vx = vx;
  b.vy = vy;
}

// Whether the robot centre (x, y) is within robot_r + r_o of the disc.
__device__ __forceinline__ bool dyn_touch(const DevCfg& c, const Obst& b, float x, float y) {
  const float dx = b.x - x, dy = b.y - y;
  return fmaf(dx, dx, dy * dy) <= c.dyn_rr2;
}

// Episode draws of disc o from the episode hash prefix pre: up to eight
// candidate centres uniform over [r_o, W - r_o] x [r_o, H - r_o] (slots
// 16 + 16 o + a; x from the top 24 bits, y from bits 16..39), the first on a
// free cell and farther than the keep-out from S and G taken (else the last);
// heading uniform in [-pi, pi) and speed uniform in [v_lo, v_hi] from slot
// 16 + 16 o + 8.
__device__ __forceinline__ Obst dyn_draw(const DevCfg& c, const MapDesc& m, const uint8_t* __restrict__ clr,
                                         const Layout& L, uint64_t pre, int o) {
  const float r = c.dyn_r;
  const float hx = (float)m.w - r, hy = (float)m.h - r;
  float px = r, py = r;
  for (int a = 0; a < 8; ++a) {
    const uint64_t hp = sm_at(pre, (uint64_t)(16 + 16 * o + a));
    px = r + u24_hi(hp) * (hx - r);
    py = r + u24_mid(hp) * (hy - r);
    const float dsx = px - L.sx, dsy = py - L.sy, dgx = px - L.gx, dgy = py - L.gy;
    const bool ok = __ldg(clr + __float2int_rd(py) * m.clr_ld + __float2int_rd(px)) != 0 &&
                    fmaf(dsx, dsx, dsy * dsy) > c.dyn_keep2 && fmaf(dgx, dgx, dgy * dgy) > c.dyn_keep2;
    if (ok) break;
  }
  const uint64_t hv = sm_at(pre, (uint64_t)(16 + 16 * o + 8));
  const float th = -kPi + u24_hi(hv) * (kPi - (-kPi));
  const float sp = c.dyn_vlo + u24_mid(hv) * (c.dyn_vhi - c.dyn_vlo);
  float sn, cs;
  f_sincos(th, sn, cs);
  Obst b;
  b.x = px;
  b.y = py;
  b.vx = sp * cs;
  b.vy = sp * sn;
  return b;
}

// The disc centres of the warp's env, held by lanes 0 .. n_dyn - 1, in every
// lane (n_dyn is warp-uniform).
__device__ __forceinline__ void gather_discs(const DevCfg& c, const Obst& b, Discs& d) {
#pragma unroll
  for (int o = 0; o < kMaxDyn; ++o)
    if (o < c.n_dyn) {
      d.x[o] = __shfl_sync(kFull, b.x, o);
      d.y[o] = __shfl_sync(kFull, b.y, o);
    }
}

// First sample k in [1, hmax) of the ray (x, y) + k delta (ux, uy) inside the
// disc centred at (ox, oy): fma(ex, ex, ey*ey) <= r_o^2 with (ex, ey) the
// sample minus the centre (the march's sample expression); hmax when none.
// Only samples near the ray-circle intersection are tested: every sample the
// rounded test accepts lies within r_o + 0.01 cells of the centre (maps up to
// 16384 cells), so it falls in the band of half-width sqrt(re^2 - d^2) around
// the projection tc of the centre (d: the centre's distance from the ray,
// re = r_o + delta + 0.25), widened by one sample on each side.
template <bool kUnitStep>
__device__ __forceinline__ int disc_first(const DevCfg& c, float x, float y, float ux, float uy, float ox, float oy,
                                          int hmax) {
  const float dx = ox - x, dy = oy - y;
  const float tc = dx * ux + dy * uy;
  const float dp = dx * uy - dy * ux;
  const float re = c.dyn_re;
  if (!(fabsf(dp) <= re)) return hmax;
  const float half = sqrtf(fmaxf(re * re - dp * dp, 0.0f));
  const float k0f = floorf((tc - half) / c.delta) - 1.0f;
  const float k1f = ceilf((tc + half) / c.delta) + 1.0f;
  const float top = (float)(hmax - 1);
  if (!(k1f >= 1.0f) || !(k0f <= top)) return hmax;
  int k = (int)fmaxf(k0f, 1.0f);
  const int k1 = (int)fminf(k1f, top);
  for (; k <= k1; ++k) {
    const float t = kUnitStep ? (float)k : (float)k * c.delta;
    const float ex = fmaf(t, ux, x) - ox;
    const float ey = fmaf(t, uy, y) - oy;
    if (fmaf(ex, ex, ey * ey) <= c.dyn_r2) return k;
  }
  return hmax;
}

// The first hit of the ray among the map hit h and the env's discs.
template <bool kUnitStep>
__device__ __forceinline__ int discs_first(const DevCfg& c, const Discs& d, float x, float y, float ux, float uy,
                                           int h) {
#pragma unroll
  for (int o = 0; o < kMaxDyn; ++o)
    if (o < c.n_dyn) h = disc_first<kUnitStep>(c, x, y, ux, uy, d.x[o], d.y[o], h);
  return h;
}

// ------------------------------------------------- per-env constants
// Quantities that do not change between the steps of one launch.
struct EnvConst {
  MapDesc m;
  const uint32_t* rows;  // this env's bit rows
  const uint8_t* clr;    // this env's clearance map
  const uint8_t* sec;    // this env's sector plane 0 (n_sec > 1)
  Layout L;
  int env, nb;
  float off0, off1;      // heading offsets of this lane's beams (lane, lane + 32)
  uint64_t nkey;         // counter-RNG prefix of the sensor noise
  uint64_t rkey;         // counter-RNG prefix of the episode draws
};

__device__ __forceinline__ EnvConst env_const(const DevCfg& c, const SimPtrs& p, int env, int lane) {
  EnvConst k;
  k.env = env;
  k.m = p.maps[p.env_map[env]];
  k.rows = p.atlas + k.m.word_off;
  k.clr = p.clr + k.m.clr_off;
  k.sec = p.sec ? p.sec + k.m.sec_off : nullptr;
  k.L = layout_of(c, k.m);
  k.nb = p.env_beams ? p.env_beams[env] : c.B;
  // beam j points at phi + j * (fov / (nb - 1)) - fov / 2
  const float stepb = c.fov / (float)(k.nb - 1);
  k.off0 = (float)lane * stepb - c.half_fov;
  k.off1 = (float)(lane + 32) * stepb - c.half_fov;
  k.nkey = sm_at(sm_at(c.seed, kStreamNoise), (uint64_t)k.env);
  k.rkey = sm_at(sm_at(c.seed, kStreamReset), (uint64_t)k.env);
  return k;
}

// ---------------------------------------------------- observation
// This lane's share of an observation row: beams lane and lane + 32, and
// entry n_beams + lane for lanes 0..4.
struct ObsRegs {
  float b0, b1, ex;
};
struct Aux {
  float min_range, alpha, ddx, ddy;
};
// Standard normal samples of this lane's beams for one (episode, step).
struct Noise {
  float n0, n1;
};

// Box-Muller on one 64-bit draw: u1 in (0, 1] from the top 24 bits, u2 in
// [0, 1) from bits 16..39; n = sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ float box_muller(uint64_t hs) {
  const float u1 = (float)((uint32_t)(hs >> 40) + 1u) * kTwoPow24Inv;
  const float u2 = u24_mid(hs);
  const float l = f_log(u1);
  const float rad = sqrtf(-2.0f * l);
  const float ang = u2 * (2.0f * kPi);
  float sn, cs;
  f_sincos(ang, sn, cs);
  return rad * cs;
}

// Noise of the observation taken at step ep_step of episode ep_id.  It does
// not depend on the scan, so it is drawn ahead, off the scan's critical path.
__device__ __forceinline__ Noise noise_for(const EnvConst& k, float sigma, uint32_t ep_id, uint32_t ep_step,
                                           int lane) {
  Noise z;
  z.n0 = 0.0f;
  z.n1 = 0.0f;
  if (sigma > 0.0f) {
    const uint64_t pre = sm_at(k.nkey, ((uint64_t)ep_id << 32) | ep_step);
    z.n0 = box_muller(sm_at(pre, (uint64_t)lane));
    if (k.nb > 32) z.n1 = box_muller(sm_at(pre, (uint64_t)(lane + 32)));
  }
  return z;
}

// Normalised range of the beam at heading offset `off` from the pose (x, y,
// phi), with noise sigma * nz; mn takes the minimum noise-free range.  With
// kDyn the discs d are in the way too.
// A beam's direction, its skip values and, where the march takes the
// unbounded loop, sample 1's skip value: issued before the noise draws of
// the scan, so that the first (usually L1-missing) load's latency hides
// behind them.
struct BeamPre {
  float ux, uy;
  const uint8_t* skip;
  int s1;  // -1: not loaded (the march starts as usual)
};
__device__ __forceinline__ BeamPre beam_pre(const DevCfg& c, const EnvConst& k, float x, float y, float phi,
                                            float off) {
  BeamPre b;
  const float beta = phi + off;
  float sn, cs;
  f_sincos(beta, sn, cs);
  b.ux = -cs;
  b.uy = -sn;
  // the skip values of this beam's sector: u = -(cos beta, sin beta) has
  // angle beta + pi, whose sector index is floor(beta n_sec / 2pi) mod n_sec
  b.skip = c.n_sec > 1 ? k.sec + (long long)(__float2int_rd(beta * c.sec_scale) & (c.n_sec - 1)) * k.m.sec_plane
                       : k.clr;
  b.s1 = -1;
  if (c.delta == 1.0f) {
    if (march_fast<true>(k.m.w, k.m.h, x, y, 1))
      b.s1 = march_skip_at<true>(b.skip, k.m.w, k.m.h, k.m.clr_ld, march_bias(k.m.clr_ld), x, y, b.ux, b.uy, c.delta, 1);
  } else if (march_fast<false>(k.m.w, k.m.h, x, y, c.skip_ok)) {
    b.s1 = march_skip_at<false>(b.skip, k.m.w, k.m.h, k.m.clr_ld, march_bias(k.m.clr_ld), x, y, b.ux, b.uy, c.delta, 1);
  }
  return b;
}

template <bool kDyn = false>
__device__ __forceinline__ float beam_at(const DevCfg& c, const EnvConst& k, float x, float y, float phi,
                                         float sigma, float off, float nz, float& mn, const Discs* d = nullptr,
                                         const BeamPre* pre = nullptr) {
  const BeamPre b = pre ? *pre : beam_pre(c, k, x, y, phi, off);
  const float ux = b.ux, uy = b.uy;
  int h = c.delta == 1.0f
              ? march<true>(b.skip, k.m.w, k.m.h, k.m.clr_ld, x, y, ux, uy, c.delta, c.kmax, 1, b.s1)
              : march<false>(b.skip, k.m.w, k.m.h, k.m.clr_ld, x, y, ux, uy, c.delta, c.kmax, c.skip_ok, b.s1);
  if (kDyn)
    h = c.delta == 1.0f ? discs_first<true>(c, *d, x, y, ux, uy, h) : discs_first<false>(c, *d, x, y, ux, uy, h);
  float r = fminf((float)h * c.delta, c.range_max);
  mn = fminf(mn, r);
  if (sigma > 0.0f) {
    // additive Gaussian sensor noise on the reported range, clamped
    r = r + sigma * nz;
    r = fminf(fmaxf(r, 0.0f), c.range_max);
  }
  return r / c.range_max;
}

template <bool kDyn = false>
__device__ __forceinline__ float beam_range(const DevCfg& c, const EnvConst& k, const Env& s, float off, float nz,
                                            float& mn, const Discs* d = nullptr) {
  return beam_at<kDyn>(c, k, s.x, s.y, s.phi, s.sigma, off, nz, mn, d);
}

// Goal in the robot frame (forward (-cos phi, -sin phi), left = forward
// turned by +90 degrees) and the heading-to-goal angle.
struct GoalFrame {
  float ddx, ddy, fwd, left, alpha;
};
__device__ __forceinline__ GoalFrame goal_frame(const Layout& L, const Env& s) {
  GoalFrame g;
  const float sn = s.sphi, cs = s.cphi;
  g.ddx = L.gx - s.x;
  g.ddy = L.gy - s.y;
  g.fwd = -(g.ddx * cs + g.ddy * sn);
  g.left = sn * g.ddx - cs * g.ddy;
  g.alpha = f_atan2(g.left, g.fwd);
  return g;
}

// Observation entry B + q (q = 0..4): fwd/D, left/D, alpha/pi, vl/v_nom,
// va/w_nom (q >= 4 gives the last).
__device__ __forceinline__ float obs_extra(const DevCfg& c, const Layout& L, const Env& s, const GoalFrame& g,
                                           int q) {
  const float num = q == 0 ? g.fwd : q == 1 ? g.left : q == 2 ? g.alpha : q == 3 ? s.vl : s.va;
  const float den = q < 2 ? L.D : q == 2 ? kPi : q == 3 ? c.v_nom : c.w_nom;
  return num / den;
}

template <bool kDyn = false>
__device__ __forceinline__ void observe(const DevCfg& c, const EnvConst& k, const Env& s, const Noise& z, int lane,
                                        ObsRegs& o, Aux& aux, const Discs* d = nullptr) {
  // independent of the scan, so issued first; lanes 0..4 hold the extras
  const GoalFrame g = goal_frame(k.L, s);
  const float ddx = g.ddx, ddy = g.ddy, alpha = g.alpha;
  o.ex = obs_extra(c, k.L, s, g, lane);
  float mn = c.range_max;
  o.b0 = lane < k.nb ? beam_range<kDyn>(c, k, s, k.off0, z.n0, mn, d) : 1.0f;
  o.b1 = lane + 32 < k.nb ? beam_range<kDyn>(c, k, s, k.off1, z.n1, mn, d) : 1.0f;
  // ranges are >= 0, so their bit patterns order like the values
  aux.min_range = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(mn)));
  aux.alpha = alpha;
  aux.ddx = ddx;
  aux.ddy = ddy;
}

__device__ __forceinline__ void write_obs(float* row, const ObsRegs& o, int B, int lane) {
  if (lane < B) row[lane] = o.b0;
  if (lane + 32 < B) row[lane + 32] = o.b1;
  if (lane < 5) row[B + lane] = o.ex;
}

// ------------------------------------------------------------ reset
__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
  const uint32_t hi = __shfl_sync(kFull, (uint32_t)(v >> 32), src);
  const uint32_t lo = __shfl_sync(kFull, (uint32_t)v, src);
  return ((uint64_t)hi << 32) | lo;
}

// The episode draws (Sec. 3.2.4) from the eight slot hashes h[0..7] of
// (seed, env, ep_id): parameters, start near S, random heading.
__device__ __forceinline__ void apply_draws(const DevCfg& c, const Layout& L, Env& s, uint32_t ep_id, uint64_t h0,
                                            uint64_t h1, uint64_t h2, uint64_t h3, uint64_t h4, uint64_t h5,
                                            uint64_t h6, uint64_t h7) {
  s.dt = c.dt_lo + u24_hi(h0) * (c.dt_hi - c.dt_lo);
  const uint32_t d = (uint32_t)c.delay_lo + (uint32_t)(h1 >> 32) % (uint32_t)c.delay_span;
  s.K = c.k_lo + u24_hi(h2) * (c.k_hi - c.k_lo);
  s.cap = c.cap_lo + u24_hi(h3) * (c.cap_hi - c.cap_lo);
  s.sigma = c.sig_lo + u24_hi(h4) * (c.sig_hi - c.sig_lo);
  const float J = c.jitter;
  const float jx = -J + u24_hi(h5) * (J - (-J));
  const float jy = -J + u24_hi(h6) * (J - (-J));
  s.x = L.sx + jx;
  s.y = L.sy + jy;
  s.phi = -kPi + u24_hi(h7) * (kPi - (-kPi));
  f_sincos(s.phi, s.sphi, s.cphi);
  s.vl = 0.0f;
  s.va = 0.0f;
  s.ep_step = 0;
  s.ep_id = ep_id;
  s.fifo = kNoAction | (kNoAction << 8) | (d << 16);
}

// New episode ep_id (Sec. 3.2.4): every randomised parameter re-drawn from
// the counter RNG keyed by (seed, env, ep_id); start near S.  Lanes 0..7
// draw one slot each.  With kDyn lane o < n_dyn draws disc o into *b and
// every lane receives the new centres in *d.
template <bool kDyn = false>
__device__ __forceinline__ void reset_env(const DevCfg& c, const EnvConst& k, Env& s, uint32_t ep_id, int lane,
                                          Obst* b = nullptr, Discs* d = nullptr) {
  const uint64_t pre = sm_at(k.rkey, (uint64_t)ep_id);
  const uint64_t mine = sm_at(pre, (uint64_t)(lane & 7));
  const uint64_t h0 = shfl_u64(mine, 0), h1 = shfl_u64(mine, 1), h2 = shfl_u64(mine, 2);
  const uint64_t h3 = shfl_u64(mine, 3), h4 = shfl_u64(mine, 4), h5 = shfl_u64(mine, 5);
  const uint64_t h6 = shfl_u64(mine, 6), h7 = shfl_u64(mine, 7);
  apply_draws(c, k.L, s, ep_id, h0, h1, h2, h3, h4, h5, h6, h7);
  if (kDyn) {
    if (lane < c.n_dyn) *b = dyn_draw(c, k.m, k.clr, k.L, pre, lane);
    gather_discs(c, *b, *d);
  }
}

// The same draws by one lane alone (the lane holds its own env): slot j of
// the episode hash is sm_at(pre, j), as reset_env's lane j computes it.
__device__ __forceinline__ void reset_env_lane(const DevCfg& c, const Layout& L, uint64_t rkey, Env& s,
                                               uint32_t ep_id) {
  const uint64_t pre = sm_at(rkey, (uint64_t)ep_id);
  apply_draws(c, L, s, ep_id, sm_at(pre, 0ull), sm_at(pre, 1ull), sm_at(pre, 2ull), sm_at(pre, 3ull),
              sm_at(pre, 4ull), sm_at(pre, 5ull), sm_at(pre, 6ull), sm_at(pre, 7ull));
}

// ------------------------------------------------------------- step
// Control delay, target velocity, Eq. 5, Eq. 6 (new velocity, old heading),
// heading wrap into [-pi, pi).
__device__ __forceinline__ bool kinematics(const DevCfg& c, Env& s, uint32_t a) {
  const uint32_t q0 = s.fifo & 0xFFu, q1 = (s.fifo >> 8) & 0xFFu, d = (s.fifo >> 16) & 0xFFu;
  const uint32_t ahat = d == 0 ? a : (d == 1 ? q0 : q1);
  s.fifo = (a & 0xFFu) | (q0 << 8) | (d << 16);
  float vhl = 0.0f, vha = 0.0f;
  if (ahat < (uint32_t)c.n_actions) {
    vhl = c.av[ahat] * s.cap;
    vha = c.aw[ahat] * s.cap;
  }
  const float omk = 1.0f - s.K;
  s.vl = s.K * s.vl + omk * vhl;
  s.va = s.K * s.va + omk * vha;
  // Eq. 6 uses the heading before the step: its sin/cos are cached in s
  s.x = s.x - s.dt * (s.vl * s.cphi);
  s.y = s.y - s.dt * (s.vl * s.sphi);
  float phi = s.phi + s.dt * s.va;
  if (phi >= kPi)
    phi = phi - 2.0f * kPi;
  else if (phi < -kPi)
    phi = phi + 2.0f * kPi;
  s.phi = phi;
  f_sincos(phi, s.sphi, s.cphi);
  s.ep_step += 1u;
  s.t += 1u;
  return a >= (uint32_t)c.n_actions;
}

struct StepOut {
  float rew;
  uint32_t done;
};

// The terms of Eq. 11 that do not need the scan, summed in order:
// ((0.3 r_d1 + 0.1 r_d2) + 0.3 r_v) + 0.3 r_alpha.
__device__ __forceinline__ float reward_partial(const DevCfg& c, const Layout& L, const Env& s, float alpha,
                                                float ddx, float ddy) {
  const float d1sq = fmaf(ddx, ddx, ddy * ddy);
  const float d1 = sqrtf(d1sq);
  const float rd1 = 1.0f - d1 / L.D;
  const float ex = L.gx - L.sx, ey = L.gy - L.sy;
  const float px = s.x - L.sx, py = s.y - L.sy;
  const float cr = ex * py - ey * px;
  const float t2 = fabsf(cr) / L.D / L.D;
  const float rd2 = 1.0f - (t2 + t2);
  const float vmax = c.v_nom * s.cap;
  const float rv = s.vl > 0.5f * vmax ? 1.0f : 0.0f;
  const float ra = 1.0f - fabsf(alpha) / kPi;
  float r = 0.3f * rd1;
  r = r + 0.1f * rd2;
  r = r + 0.3f * rv;
  r = r + 0.3f * ra;
  return r;
}

// The last term, r_d, from the scan's minimum noise-free range.
__device__ __forceinline__ float reward_finish(const DevCfg& c, float partial, float min_range) {
  const float rdn = min_range < c.near_dist ? -1.0f : 0.0f;
  return partial + 0.1f * rdn;
}

// Eq. 11 for a live (not collided, not arrived) step: 0.3 r_d1 + 0.1 r_d2 +
// 0.3 r_v + 0.3 r_alpha + 0.1 r_d at the state `s` whose scan gave `aux`.
__device__ __forceinline__ float shaped_reward(const DevCfg& c, const EnvConst& k, const Env& s, const Aux& aux) {
  return reward_finish(c, reward_partial(c, k.L, s, aux.alpha, aux.ddx, aux.ddy), aux.min_range);
}

// One full step of one env by its warp.  `term_row` (may be null) receives
// the pre-reset observation of a done env; `o` returns this lane's share of
// the observation after the step (after the reset when done).  With kDyn,
// lane o < n_dyn holds disc o in *b and every lane the centres in *d (both
// updated: motion, and the new episode's draws when done).
template <bool kDyn = false>
__device__ __forceinline__ StepOut env_step(const DevCfg& c, const SimPtrs& p, const EnvConst& k, Env& s,
                                            uint32_t a, int lane, ObsRegs& o, float* term_row, Obst* b = nullptr,
                                            Discs* d = nullptr) {
  // noise of the observation this step produces, drawn before the scan
  const Noise z = noise_for(k, s.sigma, s.ep_id, s.ep_step + 1u, lane);
  const bool bad = kinematics(c, s, a);
  if (bad && lane == 0) atomicOr(p.status, 1u);
  bool col = collide_warp(c, k.m, k.rows, k.clr, s.x, s.y, lane);
  if (kDyn) {
    // the discs move with the env's control interval before the tests
    bool touch = false;
    if (lane < c.n_dyn) {
      dyn_move(c, k.m, k.clr, s.dt, *b);
      touch = dyn_touch(c, *b, s.x, s.y);
    }
    col = __any_sync(kFull, touch) || col;
    gather_discs(c, *b, *d);
  }
  Aux aux;
  observe<kDyn>(c, k, s, z, lane, o, aux, d);
  const float d1sq = fmaf(aux.ddx, aux.ddx, aux.ddy * aux.ddy);
  const bool arrive = d1sq <= c.goal_r * c.goal_r;
  const bool trunc = s.ep_step >= (uint32_t)c.t_max;
  float r = shaped_reward(c, k, s, aux);
  if (col)
    r = -10.0f;
  else if (arrive)
    r = 75.0f;
  StepOut out;
  out.rew = r;
  out.done = (col ? 1u : 0u) | (arrive ? 2u : 0u) | (trunc ? 4u : 0u);
  if (out.done) {
    // AutoReset (Sec. 3.2.5): keep s' for the caller, then a new episode
    if (term_row) write_obs(term_row, o, c.B, lane);
    reset_env<kDyn>(c, k, s, s.ep_id + 1u, lane, b, d);
    const Noise z0 = noise_for(k, s.sigma, s.ep_id, 0u, lane);
    observe<kDyn>(c, k, s, z0, lane, o, aux, d);
  }
  return out;
}

// The part of a step that the next step depends on: delay, Eq. 5, Eq. 6,
// collision, arrival, truncation and, when done, the AutoReset draws.  It
// never needs the LiDAR.  `pre` receives the state after the motion and
// before the reset.  Returns the done flags.
__device__ __forceinline__ uint32_t pose_step(const DevCfg& c, const SimPtrs& p, const EnvConst& k, Env& s, Env& pre,
                                              uint32_t a, int lane, bool report) {
  const bool bad = kinematics(c, s, a);
  if (bad && report && lane == 0) atomicOr(p.status, 1u);
  const bool col = collide_warp(c, k.m, k.rows, k.clr, s.x, s.y, lane);
  const float ddx = k.L.gx - s.x, ddy = k.L.gy - s.y;
  const float d1sq = fmaf(ddx, ddx, ddy * ddy);
  const bool arrive = d1sq <= c.goal_r * c.goal_r;
  const bool trunc = s.ep_step >= (uint32_t)c.t_max;
  const uint32_t done = (col ? 1u : 0u) | (arrive ? 2u : 0u) | (trunc ? 4u : 0u);
  pre = s;
  if (done) reset_env(c, k, s, s.ep_id + 1u, lane);
  return done;
}

// The rest of a step, given pose_step's result: the observation (after the
// reset when done) and the reward (from the pre-reset scan when the episode
// was only truncated; the terminal constants otherwise).
__device__ __forceinline__ float obs_step(const DevCfg& c, const EnvConst& k, const Env& s, const Env& pre,
                                          uint32_t done, int lane, ObsRegs& o) {
  Aux aux;
  float r;
  if (done & 1u) {
    r = -10.0f;
  } else if (done & 2u) {
    r = 75.0f;
  } else if (done) {
    const Noise zp = noise_for(k, pre.sigma, pre.ep_id, pre.ep_step, lane);
    observe(c, k, pre, zp, lane, o, aux);
    r = shaped_reward(c, k, pre, aux);
  }
  const Noise z = noise_for(k, s.sigma, s.ep_id, s.ep_step, lane);
  observe(c, k, s, z, lane, o, aux);
  if (!done) r = shaped_reward(c, k, s, aux);
  return r;
}

// Random action of step t for env (uniform over the action table): lane l
// draws the action of step t0 + l, so that one batch of hashes serves 32 steps.
__device__ __forceinline__ uint32_t random_action_for(const DevCfg& c, uint64_t akey, uint32_t t) {
  const uint64_t ha = sm_at(sm_at(akey, (uint64_t)t), 0ull);
  return (uint32_t)(ha >> 32) % (uint32_t)c.n_actions;
}

// ------------------------------------------------- lane-parallel step
struct __align__(16) StepScanRec {
  float ax, ay, aphi, asigma;  // post-motion state (scan A)
  uint32_t anlo, anhi;         // its noise key
  float rpart;                 // scan-free part of Eq. 11 at the post-motion state
  uint32_t done;
  float exa[5];                // observation entries B .. B + 4 of scan A
  float bx, by, bphi;          // reset state (scan B, done envs)
  float bsigma;
  uint32_t bnlo, bnhi;
  int map, nb;
  float exb[5];                // observation entries of scan B
  float stepb;                 // beam spacing of the env
  int env;
  int pad[3];
};
static_assert(sizeof(StepScanRec) == 128, "step scan record is eight 16-byte words");

// Scan of one pose by the warp for an env of map m with nb beams: this
// lane's normalised ranges into b0 / b1; returns the minimum noise-free range.
// kPre: the first beam's first march load is issued before the noise draws
// (beam_pre); the kernels with little register room leave it off.
template <bool kDyn = false, bool kPre = false>
__device__ __forceinline__ float scan_env(const DevCfg& c, const SimPtrs& p, const MapDesc& m, int nb, float stepb,
                                          float x, float y, float phi, float sigma, uint64_t nk, int lane,
                                          float& b0, float& b1, const Discs* d = nullptr) {
  EnvConst k;
  k.m = m;
  k.clr = p.clr + m.clr_off;
  k.sec = p.sec ? p.sec + m.sec_off : nullptr;
  k.nb = nb;
  const float off0 = (float)lane * stepb - c.half_fov;
  const float off1 = (float)(lane + 32) * stepb - c.half_fov;
  BeamPre p0;
  if (kPre && lane < nb) p0 = beam_pre(c, k, x, y, phi, off0);
  float n0 = 0.0f, n1 = 0.0f;
  if (sigma > 0.0f) {
    n0 = box_muller(sm_at(nk, (uint64_t)lane));
    if (nb > 32) n1 = box_muller(sm_at(nk, (uint64_t)(lane + 32)));
  }
  float mn = c.range_max;
  b0 = lane < nb ? beam_at<kDyn>(c, k, x, y, phi, sigma, off0, n0, mn, d, kPre ? &p0 : nullptr) : 1.0f;
  b1 = lane + 32 < nb ? beam_at<kDyn>(c, k, x, y, phi, sigma, off1, n1, mn, d) : 1.0f;
  return __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(mn)));
}

__device__ __forceinline__ void write_row(float* row, float b0, float b1, const float* ex, int B, int lane) {
  if (lane < B) row[lane] = b0;
  if (lane + 32 < B) row[lane + 32] = b1;
  if (lane < 5) row[B + lane] = ex[lane];
}


// The scan-free part of the observation of env i at its current state s (one
// lane), into the scan-A fields of r: the first observation of a rollout
// whose steps run lane_step.
__device__ __forceinline__ void lane_observe(const DevCfg& c, const SimPtrs& p, int i, const Env& s,
                                             StepScanRec& r) {
  const int mid = p.env_map[i];
  const MapDesc m = p.maps[mid];
  const Layout L = layout_of(c, m);
  const int nb = p.env_beams ? p.env_beams[i] : c.B;
  const uint64_t nkey = sm_at(sm_at(c.seed, kStreamNoise), (uint64_t)i);
  const GoalFrame g = goal_frame(L, s);
  const uint64_t nka = sm_at(nkey, ((uint64_t)s.ep_id << 32) | s.ep_step);
  r.ax = s.x, r.ay = s.y, r.aphi = s.phi, r.asigma = s.sigma;
  r.anlo = (uint32_t)nka, r.anhi = (uint32_t)(nka >> 32);
  for (int q = 0; q < 5; ++q) r.exa[q] = obs_extra(c, L, s, g, q);
  r.rpart = 0.0f;
  r.done = 0u;
  r.map = mid;
  r.env = i;
  r.nb = nb;
  r.stepb = c.fov / (float)(nb - 1);
}

// One step of one env per lane (sg_sim_step and the fused Q-net rollout):
// delay, Eq. 5, Eq. 6, the collision test (map bounds and clearance per lane,
// the bit rows for the envs that need them with the whole warp), arrival,
// truncation, the AutoReset draws, and everything of the observation and of
// Eq. 11 that does not need a scan, into the env's record r (scan A: the
// post-motion state; scan B: the reset state of a done env).  s: the env's
// state in, the state after the step out.  Lanes with live = false take part
// in the warp-wide collision tests only.  With kDyn the env's discs move
// (and collide) here too; their centres for scan A go to da, those of the
// reset state to db, and the discs' new state to global memory.  Returns the
// done flags.
template <bool kDyn = false>
__device__ __forceinline__ uint32_t lane_step(const DevCfg& c, const SimPtrs& p, int i, bool live, Env& s,
                                              uint32_t a, StepScanRec& r, int lane, Discs* da = nullptr,
                                              Discs* db = nullptr) {
  MapDesc m;
  Layout L;
  int mid = 0, nb = c.B;
  uint32_t d = 0;
  bool slow = false;
  if (live) {
    mid = p.env_map[i];
    m = p.maps[mid];
    L = layout_of(c, m);
    nb = p.env_beams ? p.env_beams[i] : c.B;
    if (kinematics(c, s, a)) atomicOr(p.status, 1u);
    if (s.x < 0.0f || s.y < 0.0f || s.x >= (float)m.w || s.y >= (float)m.h) {
      d = 1u;
    } else {
      const int own = __ldg(p.clr + m.clr_off + __float2int_rd(s.y) * m.clr_ld + __float2int_rd(s.x));
      slow = own < c.clr_collide;
    }
    const float ddx = L.gx - s.x, ddy = L.gy - s.y;
    if (fmaf(ddx, ddx, ddy * ddy) <= c.goal_r * c.goal_r) d |= 2u;
    if (s.ep_step >= (uint32_t)c.t_max) d |= 4u;
    if (kDyn) {
      const uint8_t* clr = p.clr + m.clr_off;
      for (int o = 0; o < c.n_dyn; ++o) {
        Obst b = load_obst(p, o, i);
        dyn_move(c, m, clr, s.dt, b);
        if (dyn_touch(c, b, s.x, s.y)) d |= 1u;
        da->x[o] = b.x;
        da->y[o] = b.y;
        store_obst(p, o, i, b);
      }
    }
  }
  // collision tests that need the bit rows, one env at a time
  unsigned sm = __ballot_sync(kFull, slow);
  while (sm) {
    const int e = __ffs(sm) - 1;
    sm &= sm - 1u;
    const MapDesc me = p.maps[__shfl_sync(kFull, mid, e)];
    const float xe = __shfl_sync(kFull, live ? s.x : 0.0f, e), ye = __shfl_sync(kFull, live ? s.y : 0.0f, e);
    if (collide_rows_warp(c, me, p.atlas + me.word_off, xe, ye, lane) && lane == e) d |= 1u;
  }
  if (live) {
    const uint64_t nkey = sm_at(sm_at(c.seed, kStreamNoise), (uint64_t)i);
    const GoalFrame g = goal_frame(L, s);
    const uint64_t nka = sm_at(nkey, ((uint64_t)s.ep_id << 32) | s.ep_step);
    r.ax = s.x, r.ay = s.y, r.aphi = s.phi, r.asigma = s.sigma;
    r.anlo = (uint32_t)nka, r.anhi = (uint32_t)(nka >> 32);
    for (int q = 0; q < 5; ++q) r.exa[q] = obs_extra(c, L, s, g, q);
    r.rpart = (d & 3u) ? 0.0f : reward_partial(c, L, s, g.alpha, g.ddx, g.ddy);
    r.done = d;
    r.map = mid;
    r.env = i;
    r.nb = nb;
    r.stepb = c.fov / (float)(nb - 1);
    if (d) {
      // AutoReset (Sec. 3.2.5): a new episode, observed at its step 0
      const uint64_t rkey = sm_at(sm_at(c.seed, kStreamReset), (uint64_t)i);
      reset_env_lane(c, L, rkey, s, s.ep_id + 1u);
      if (kDyn) {
        const uint64_t pre = sm_at(rkey, (uint64_t)s.ep_id);
        for (int o = 0; o < c.n_dyn; ++o) {
          const Obst b = dyn_draw(c, m, p.clr + m.clr_off, L, pre, o);
          db->x[o] = b.x;
          db->y[o] = b.y;
          store_obst(p, o, i, b);
        }
      }
      const GoalFrame gb = goal_frame(L, s);
      const uint64_t nkb = sm_at(nkey, ((uint64_t)s.ep_id << 32) | s.ep_step);
      r.bx = s.x, r.by = s.y, r.bphi = s.phi, r.bsigma = s.sigma;
      r.bnlo = (uint32_t)nkb, r.bnhi = (uint32_t)(nkb >> 32);
      for (int q = 0; q < 5; ++q) r.exb[q] = obs_extra(c, L, s, gb, q);
    }
  }
  return d;
}

}  // namespace sg
