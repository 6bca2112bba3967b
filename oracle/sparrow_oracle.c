/*
 * sparrow_oracle.c -- plain CPU oracle of the vectorized Sparrow environment
 * step (paper arxiv 2305.04180, Sec. 3.2 "Sparrow simulator").
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library.  The CUDA path never
 * includes, links or calls it, and this file includes nothing of the CUDA
 * path: the two are written separately from the same reading of the paper.
 *
 * The file is compiled twice:
 *   ORC_F32 (default) -- every real is an IEEE float, no contraction
 *            (-ffp-contract=off), fmaf() only where the step says "fma".
 *            The paper's simulator keeps its world matrix in torch tensors,
 *            whose default dtype is float32, so this is the precision that
 *            takes the discrete decisions (hit index, collision, arrival).
 *            sin/cos/atan2/log are this file's own float routines (below),
 *            written from their Taylor / atanh series, so that a float
 *            implementation elsewhere can be compared bit for bit.
 *   ORC_F64 -- every real is a double and sin/cos/atan2/log come from libm.
 *            This is the exact-math reference for the tolerance checks.
 *
 * Everything is a loop over envs, beams and march samples, in the order the
 * step is defined, with no blocking or reordering.
 *
 * Passages followed:
 *   Eq. 5 / Eq. 7   velocity update  v <- K v + (1-K) v_hat
 *   Eq. 6 / Eq. 8   pose update with the new velocity and the old heading,
 *                   motion along (-cos phi, -sin phi)
 *   Sec. 3.2        LiDAR by ray casting on the occupancy grid, sensor noise,
 *                   collision detection, AutoReset, vectorized diversity
 *   Sec. 4.3.1      5-action table, reward Eq. 11 (-10 collide, +75 arrive)
 *   sim-parameter table: K 0.6, control interval 0.1 s, delay 0.1 s,
 *                   18 cm/s, 1 rad/s, noise 1 cm
 *   Sec. 5          dynamic obstacles, named in the conclusion as the
 *                   simulator's next capability; optional (n_dyn = 0 leaves the step as above)
 * Readings where the paper is silent (beam layout, march, collision disc,
 * delay FIFO, d1/d2/alpha, random numbers) are listed in the design notes;
 * each is restated at the point of use below.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef ORC_F64
typedef double R;
#define FMA(a, b, c) fma((a), (b), (c))
#define SQRT(a) sqrt(a)
#define FLOOR(a) floor(a)
#define FABS(a) fabs(a)
#define RMIN(a, b) fmin((a), (b))
#define RMAX(a, b) fmax((a), (b))
#define PI_R 3.14159265358979323846
#else
typedef float R;
#define FMA(a, b, c) fmaf((a), (b), (c))
#define SQRT(a) sqrtf(a)
#define FLOOR(a) floorf(a)
#define FABS(a) fabsf(a)
#define RMIN(a, b) fminf((a), (b))
#define RMAX(a, b) fmaxf((a), (b))
#define PI_R 3.14159265358979323846f
#endif

#define NONE_ACTION 255u

/* random-number streams (counter-based, see orc_rng) */
#define STREAM_RESET 1u
#define STREAM_NOISE 2u
#define STREAM_ACTION 3u

typedef struct {
  int32_t n_beams; /* B_max; an observation row holds B_max + 5 reals */
  int32_t n_actions;
  int32_t t_max;
  int32_t delay_lo, delay_hi;
  int32_t n_dyn;   /* dynamic obstacles per env, 0..8 (0: none) */
  double fov, range_max, march_step, robot_radius, goal_radius, near_dist;
  double start_offset, start_jitter;
  double dt_lo, dt_hi, k_lo, k_hi, cap_lo, cap_hi, sigma_lo, sigma_hi;
  double v_nom, w_nom;
  double action_v[8], action_w[8];
  uint64_t seed;
  double dyn_radius;                 /* obstacle disc radius, cells */
  double dyn_speed_lo, dyn_speed_hi; /* obstacle speed range, cells / s */
  double dyn_keepout;                /* no obstacle starts this close to S or G */
} orc_config;

typedef struct {
  int32_t n_maps;
  int32_t pad0;
  const int32_t* w;
  const int32_t* h;
  const int64_t* off;    /* start of map m in grids */
  const uint8_t* grids;  /* grid[cy * w + cx], nonzero = occupied */
} orc_maps;

typedef struct {
  int32_t n_envs;
  int32_t pad0;
  const int32_t* env_map;
  const int32_t* env_beams; /* may be NULL: every env uses n_beams */
  R* f;        /* [9][n]: x y phi vl va dt K cap sigma */
  uint32_t* u; /* [2][n]: ep_step ep_id */
  uint8_t* b;  /* [3][n]: q0 (last action) q1 (the one before) delay */
  R* dyn;      /* [4 n_dyn][n]: obstacle o at rows 4o..4o+3 (x y vx vy); NULL when n_dyn = 0 */
} orc_envs;

enum { F_X, F_Y, F_PHI, F_VL, F_VA, F_DT, F_K, F_CAP, F_SIGMA, F_COUNT };
enum { U_STEP, U_EPID };
enum { B_Q0, B_Q1, B_DELAY };

/* ------------------------------------------------------------------ RNG */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the generator's state after
 * c+1 increments of the golden gamma is s + (c+1)*gamma, and its output is the
 * finalizer of that state.  Nesting this "value at counter c" map gives a
 * counter-based hash of several 64-bit words. */
static uint64_t sm_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t sm_at(uint64_t s, uint64_t c) {
  return sm_mix(s + (c + 1u) * 0x9E3779B97F4A7C15ULL);
}
/* the generator's output after c+1 steps from state s (exported for the pin
 * against the published sequence) */
uint64_t orc_splitmix_at(uint64_t s, uint64_t c) { return sm_at(s, c); }
uint64_t orc_rng(uint64_t seed, uint64_t stream, uint64_t env, uint64_t a, uint64_t b) {
  return sm_at(sm_at(sm_at(sm_at(seed, stream), env), a), b);
}
/* top 24 bits as a uniform in [0, 1) (exact in float) */
static R u24(uint64_t h) { return (R)(h >> 40) * (R)5.9604644775390625e-08; }
/* bits 16..39 as a second uniform in [0, 1) */
static R u24b(uint64_t h) { return (R)((h >> 16) & 0xFFFFFFu) * (R)5.9604644775390625e-08; }

/* ------------------------------------------------- elementary functions */
#ifdef ORC_F64
static void sincos_r(R a, R* s, R* c) { *s = sin(a); *c = cos(a); }
static R atan2_r(R y, R x) { return atan2(y, x); }
static R log_r(R x) { return log(x); }
#else
/* sin/cos: reduce by the nearest multiple q of pi/2 (Cody & Waite, with the
 * two-word split of pi/2 applied through fma), then the Taylor series of sin
 * to degree 11 and of cos to degree 12 on the reduced argument, with
 * coefficients (-1)^k / n!, and pick the quadrant from q mod 4. */
static void sincos_r(float a, float* s, float* c) {
  float q = rintf(a * 0.636619772f);
  int qi = (int)q;
  float r = fmaf(-q, 1.57079637050628662109375f, a);
  r = fmaf(-q, -4.371139000186243e-08f, r);
  float z = r * r;
  float ps = fmaf(z, -2.505210838544172e-08f, 2.7557319223985893e-06f);
  ps = fmaf(z, ps, -1.984126984126984e-04f);
  ps = fmaf(z, ps, 8.333333333333333e-03f);
  ps = fmaf(z, ps, -1.6666666666666666e-01f);
  float sr = fmaf(r * z, ps, r);
  float pc = fmaf(z, 2.08767569878681e-09f, -2.755731922398589e-07f);
  pc = fmaf(z, pc, 2.48015873015873e-05f);
  pc = fmaf(z, pc, -1.388888888888889e-03f);
  pc = fmaf(z, pc, 4.1666666666666664e-02f);
  pc = fmaf(z, pc, -0.5f);
  float cr = fmaf(z, pc, 1.0f);
  switch (qi & 3) {
    case 0: *s = sr; *c = cr; break;
    case 1: *s = cr; *c = -sr; break;
    case 2: *s = -sr; *c = -cr; break;
    default: *s = -cr; *c = sr; break;
  }
}

/* Coefficient literals are the float nearest to 1/n (written out so that the
 * value does not depend on how a compiler folds a constant division). */

/* atan2: octant reduction to t = min/max in [0, 1]; for t > tan(pi/8) use
 * atan t = pi/4 + atan((t-1)/(t+1)); Taylor series of atan to degree 21 on
 * |t'| <= tan(pi/8); then undo the octant. */
static float atan2_r(float y, float x) {
  float ax = fabsf(x), ay = fabsf(y);
  if (ax == 0.0f && ay == 0.0f) return 0.0f;
  int swap = ay > ax;
  float num = swap ? ax : ay;
  float den = swap ? ay : ax;
  float t = num / den;
  float base = 0.0f;
  if (t > 0.414213562373095f) {
    t = (t - 1.0f) / (t + 1.0f);
    base = 0.785398163397448f;
  }
  float w = t * t;
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

/* log: x = m * 2^e with m in (sqrt(1/2), sqrt(2)]; ln m = 2 atanh(z),
 * z = (m-1)/(m+1), atanh series to z^13; add e*ln2 in two words. */
static float log_r(float x) {
  uint32_t bits;
  memcpy(&bits, &x, 4);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  uint32_t mb = (bits & 0x7FFFFFu) | 0x3F800000u;
  float m;
  memcpy(&m, &mb, 4);
  if (m > 1.41421356237310f) {
    m = m * 0.5f;
    e = e + 1;
  }
  float z = (m - 1.0f) / (m + 1.0f);
  float w = z * z;
  float p = fmaf(w, 0.07692308f, 0.09090909f);
  p = fmaf(w, p, 0.11111111f);
  p = fmaf(w, p, 0.14285715f);
  p = fmaf(w, p, 0.2f);
  p = fmaf(w, p, 0.33333334f);
  p = fmaf(w, p, 1.0f);
  float t = z * p;
  float lnm = t + t;
  float ef = (float)e;
  float lo = fmaf(ef, 1.4286068203094172e-06f, lnm);
  return fmaf(ef, 0.693145751953125f, lo);
}
#endif

/* exported for the tests that pin these routines */
void orc_sincos(R a, R* s, R* c) { sincos_r(a, s, c); }
R orc_atan2(R y, R x) { return atan2_r(y, x); }
R orc_log(R x) { return log_r(x); }

/* ----------------------------------------------------------- map access */
static int occupied(const orc_maps* m, int32_t map, int64_t cx, int64_t cy) {
  int32_t w = m->w[map], h = m->h[map];
  if (cx < 0 || cy < 0 || cx >= w || cy >= h) return 1; /* outside = wall */
  return m->grids[m->off[map] + cy * (int64_t)w + cx] != 0;
}

/* Bit-packed copy of one grid: row stride `row_words` 32-bit words, bit
 * (cx & 31) of word (cx >> 5) holds cell cx (lowest x in the lowest bit). */
void orc_pack_map(const uint8_t* grid, int32_t w, int32_t h, int32_t row_words, uint32_t* out) {
  for (int32_t cy = 0; cy < h; ++cy)
    for (int32_t wd = 0; wd < row_words; ++wd) {
      uint32_t word = 0;
      for (int32_t bit = 0; bit < 32; ++bit) {
        int32_t cx = wd * 32 + bit;
        if (cx < w && grid[(int64_t)cy * w + cx]) word |= 1u << bit;
      }
      out[(int64_t)cy * row_words + wd] = word;
    }
}

/* ---------------------------------------------------------------- LiDAR */
/* March one beam from (x, y) along unit direction (ux, uy): samples
 * p_k = (fma(kD, ux, x), fma(kD, uy, y)) for k = 1..kmax; the first sample
 * whose cell floor(p) is occupied or outside the map is the hit.  Returns the
 * hit index, or kmax + 1 when no sample hits. */
static uint64_t g_samples = 0; /* march samples evaluated (instrumentation) */
uint64_t orc_march_samples(void) { return g_samples; }
void orc_reset_march_samples(void) { g_samples = 0; }

/* Sample point k of a ray lies in obstacle disc (ox, oy) of radius r when
 * fma(ex, ex, ey*ey) <= r*r with (ex, ey) = sample - centre. */
static int in_disc(R px, R py, R ox, R oy, R r2) {
  R ex = px - ox, ey = py - oy;
  return FMA(ex, ex, ey * ey) <= r2;
}

/* discs: nd obstacle centres as (x, y) pairs; a sample inside one is a hit */
static int32_t march(const orc_maps* m, int32_t map, const R* discs, int32_t nd, R r2, R x, R y, R ux, R uy,
                     R delta, int32_t kmax) {
  for (int32_t k = 1; k <= kmax; ++k) {
    ++g_samples;
    R t = (R)k * delta;
    R px = FMA(t, ux, x);
    R py = FMA(t, uy, y);
    R fx = FLOOR(px), fy = FLOOR(py);
    if (fx < (R)0 || fy < (R)0 || fx >= (R)m->w[map] || fy >= (R)m->h[map]) return k;
    if (occupied(m, map, (int64_t)fx, (int64_t)fy)) return k;
    for (int32_t o = 0; o < nd; ++o)
      if (in_disc(px, py, discs[2 * o], discs[2 * o + 1], r2)) return k;
  }
  return kmax + 1;
}

static int32_t kmax_of(const orc_config* c) {
  return (int32_t)FLOOR((R)c->range_max / (R)c->march_step);
}

/* Beam j of nb over the field of view, centred on the heading:
 * offset_j = j * (fov / (nb - 1)) - fov / 2 (both ends included). */
static R beam_offset(const orc_config* c, int32_t j, int32_t nb) {
  R fov = (R)c->fov;
  R half = fov * (R)0.5;
  R stepb = fov / (R)(nb - 1);
  return (R)j * stepb - half;
}

/* Ranges of nb beams from pose (x, y, phi) with nd obstacle discs (centres
 * as (x, y) pairs, radius dyn_radius) in the way; writes hit indices and
 * noise-free ranges min(h * delta, range_max). */
void orc_lidar_dyn(const orc_config* c, const orc_maps* m, int32_t map, const R* discs, int32_t nd, R x, R y,
                   R phi, int32_t nb, int32_t* hits, R* ranges) {
  R delta = (R)c->march_step, rmax = (R)c->range_max;
  R rd = (R)c->dyn_radius;
  R r2 = rd * rd;
  int32_t kmax = kmax_of(c);
  for (int32_t j = 0; j < nb; ++j) {
    R beta = phi + beam_offset(c, j, nb);
    R s, co;
    sincos_r(beta, &s, &co);
    int32_t h = march(m, map, discs, nd, r2, x, y, -co, -s, delta, kmax);
    hits[j] = h;
    ranges[j] = RMIN((R)h * delta, rmax);
  }
}

/* The same without obstacles. */
void orc_lidar(const orc_config* c, const orc_maps* m, int32_t map, R x, R y, R phi, int32_t nb,
               int32_t* hits, R* ranges) {
  orc_lidar_dyn(c, m, map, 0, 0, x, y, phi, nb, hits, ranges);
}

/* --------------------------------------------------------- collision */
/* The robot is a disc of radius r: it collides when its centre leaves the map
 * or when the centre of an occupied cell lies within r of (x, y), i.e.
 * fma(dx, dx, dy*dy) <= r*r with dx = (cx + 0.5) - x, dy = (cy + 0.5) - y. */
int32_t orc_collide(const orc_config* c, const orc_maps* m, int32_t map, R x, R y) {
  int32_t w = m->w[map], h = m->h[map];
  if (x < (R)0 || y < (R)0 || x >= (R)w || y >= (R)h) return 1;
  R r = (R)c->robot_radius;
  R r2 = r * r;
  int64_t cx0 = (int64_t)FLOOR(x - r) - 1, cx1 = (int64_t)FLOOR(x + r) + 1;
  int64_t cy0 = (int64_t)FLOOR(y - r) - 1, cy1 = (int64_t)FLOOR(y + r) + 1;
  if (cx0 < 0) cx0 = 0;
  if (cy0 < 0) cy0 = 0;
  if (cx1 > w - 1) cx1 = w - 1;
  if (cy1 > h - 1) cy1 = h - 1;
  for (int64_t cy = cy0; cy <= cy1; ++cy)
    for (int64_t cx = cx0; cx <= cx1; ++cx) {
      if (!occupied(m, map, cx, cy)) continue;
      R dx = ((R)cx + (R)0.5) - x;
      R dy = ((R)cy + (R)0.5) - y;
      R d2 = FMA(dx, dx, dy * dy);
      if (d2 <= r2) return 1;
    }
  return 0;
}

/* --------------------------------------------------------- geometry */
typedef struct {
  R sx, sy, gx, gy, D;
} layout_t;

/* Start S and goal G of a w x h map (lower-left to upper-right) and the
 * planning distance D = |G - S|. */
static layout_t layout_of(const orc_config* c, const orc_maps* m, int32_t map) {
  layout_t L;
  R off = (R)c->start_offset;
  L.sx = off;
  L.sy = off;
  L.gx = (R)m->w[map] - off;
  L.gy = (R)m->h[map] - off;
  R ex = L.gx - L.sx, ey = L.gy - L.sy;
  L.D = SQRT(FMA(ex, ex, ey * ey));
  return L;
}

static int32_t beams_of(const orc_config* c, const orc_envs* e, int32_t i) {
  return e->env_beams ? e->env_beams[i] : c->n_beams;
}

/* Observation of env i at its current state (Sec. 4.3.1 state, normalised and
 * relative): nb noisy ranges / range_max (rows padded to n_beams with 1.0),
 * then goal in the robot frame / D (forward, left), alpha / pi, vl / v_nom,
 * va / w_nom.  Returns the smallest noise-free range and fills alpha and the
 * goal vector for the reward. */
typedef struct {
  R min_range, alpha, ddx, ddy;
} obs_aux;

static obs_aux observe(const orc_config* c, const orc_maps* m, const orc_envs* e, int32_t i, R* obs) {
  int32_t n = e->n_envs;
  int32_t map = e->env_map[i];
  int32_t nb = beams_of(c, e, i);
  int32_t B = c->n_beams;
  R x = e->f[F_X * n + i], y = e->f[F_Y * n + i], phi = e->f[F_PHI * n + i];
  R sigma = e->f[F_SIGMA * n + i];
  uint32_t ep_step = e->u[U_STEP * n + i], ep_id = e->u[U_EPID * n + i];
  R rmax = (R)c->range_max;
  int32_t hits[64];
  R ranges[64];
  R discs[16];
  int32_t nd = c->n_dyn;
  for (int32_t o = 0; o < nd; ++o) {
    discs[2 * o] = e->dyn[(4 * o + 0) * n + i];
    discs[2 * o + 1] = e->dyn[(4 * o + 1) * n + i];
  }
  orc_lidar_dyn(c, m, map, discs, nd, x, y, phi, nb, hits, ranges);
  obs_aux aux;
  aux.min_range = rmax;
  for (int32_t j = 0; j < nb; ++j) aux.min_range = RMIN(aux.min_range, ranges[j]);
  /* sensor noise: additive Gaussian (Box-Muller from one 64-bit draw) on the
   * reported range only, clamped to [0, range_max] */
  for (int32_t j = 0; j < nb; ++j) {
    R rj = ranges[j];
    if (sigma > (R)0) {
      uint64_t hsh = orc_rng(c->seed, STREAM_NOISE, (uint64_t)i,
                             ((uint64_t)ep_id << 32) | ep_step, (uint64_t)j);
      R u1 = (R)((hsh >> 40) + 1u) * (R)5.9604644775390625e-08; /* (0, 1] */
      R u2 = u24b(hsh);                                          /* [0, 1) */
      R l = log_r(u1);
      R rad = SQRT((R)-2 * l);
      R ang = u2 * ((R)2 * PI_R);
      R sn, cs;
      sincos_r(ang, &sn, &cs);
      R nz = rad * cs;
      rj = rj + sigma * nz;
      rj = RMIN(RMAX(rj, (R)0), rmax);
    }
    obs[j] = rj / rmax;
  }
  for (int32_t j = nb; j < B; ++j) obs[j] = (R)1;
  layout_t L = layout_of(c, m, map);
  R s, co;
  sincos_r(phi, &s, &co);
  R ddx = L.gx - x, ddy = L.gy - y;
  /* heading direction u = (-cos phi, -sin phi) (Eq. 6); left = u rotated +90 */
  R fwd = -(ddx * co + ddy * s);
  R left = s * ddx - co * ddy;
  R alpha = atan2_r(left, fwd);
  obs[B + 0] = fwd / L.D;
  obs[B + 1] = left / L.D;
  obs[B + 2] = alpha / PI_R;
  obs[B + 3] = e->f[F_VL * n + i] / (R)c->v_nom;
  obs[B + 4] = e->f[F_VA * n + i] / (R)c->w_nom;
  aux.alpha = alpha;
  aux.ddx = ddx;
  aux.ddy = ddy;
  return aux;
}

/* ------------------------------------------------ dynamic obstacles */
/* The paper leaves dynamic obstacles to future work (Sec. 5).  Reading used
 * here: each env has n_dyn discs of radius r_o moving in straight lines at a
 * constant speed, re-drawn at every episode start like the other randomised
 * parameters.  Per step, after the robot's motion, each disc advances by
 * dt * v (the env's control interval); a centre that leaves [r_o, W - r_o]
 * (resp. H) is mirrored back into it and that velocity component changes
 * sign; a centre that would enter an occupied cell stays where it was and
 * the velocity is reversed.  The robot collides with a disc when the centres
 * are within robot_radius + r_o (fma(dx,dx,dy*dy) <= (r + r_o)^2), and the
 * LiDAR sees the discs (a march sample inside a disc is a hit). */

/* Mirror coordinate v into [lo, hi]; flips *vel when it mirrors. */
static R dyn_reflect(R v, R lo, R hi, R* vel) {
  if (v < lo) {
    v = lo + (lo - v);
    *vel = -*vel;
  } else if (v > hi) {
    v = hi - (v - hi);
    *vel = -*vel;
  }
  return RMIN(RMAX(v, lo), hi);
}

/* One step of obstacle o of env i with control interval dt. */
static void dyn_move(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i, int32_t o, R dt) {
  int32_t n = e->n_envs, map = e->env_map[i];
  R* ox = &e->dyn[(4 * o + 0) * n + i];
  R* oy = &e->dyn[(4 * o + 1) * n + i];
  R* vx = &e->dyn[(4 * o + 2) * n + i];
  R* vy = &e->dyn[(4 * o + 3) * n + i];
  R r = (R)c->dyn_radius;
  R hx = (R)m->w[map] - r, hy = (R)m->h[map] - r;
  R nvx = *vx, nvy = *vy;
  R nx = *ox + dt * nvx;
  R ny = *oy + dt * nvy;
  nx = dyn_reflect(nx, r, hx, &nvx);
  ny = dyn_reflect(ny, r, hy, &nvy);
  if (occupied(m, map, (int64_t)FLOOR(nx), (int64_t)FLOOR(ny))) {
    *vx = -*vx;
    *vy = -*vy;
    return;
  }
  *ox = nx;
  *oy = ny;
  *vx = nvx;
  *vy = nvy;
}

/* Whether the robot at (x, y) touches one of env i's discs. */
static int dyn_collide(const orc_config* c, const orc_envs* e, int32_t i, R x, R y) {
  int32_t n = e->n_envs;
  R rr = (R)c->robot_radius + (R)c->dyn_radius;
  R rr2 = rr * rr;
  for (int32_t o = 0; o < c->n_dyn; ++o) {
    R dx = e->dyn[(4 * o + 0) * n + i] - x;
    R dy = e->dyn[(4 * o + 1) * n + i] - y;
    if (FMA(dx, dx, dy * dy) <= rr2) return 1;
  }
  return 0;
}

/* Episode draws of obstacle o: up to 8 candidate centres, uniform over
 * [r_o, W - r_o] x [r_o, H - r_o] from slots 16 + 16 o + a of the episode
 * hash (x from the top 24 bits, y from bits 16..39); the first one on a free
 * cell and farther than dyn_keepout from S and from G is taken (the last one
 * when none is).  Heading uniform in [-pi, pi) and speed uniform in
 * [speed_lo, speed_hi] from slot 16 + 16 o + 8. */
static void dyn_draw(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i, uint32_t ep_id, int32_t o,
                     R sx, R sy, R gx, R gy) {
  int32_t n = e->n_envs, map = e->env_map[i];
  R r = (R)c->dyn_radius;
  R hx = (R)m->w[map] - r, hy = (R)m->h[map] - r;
  R kp = (R)c->dyn_keepout;
  R keep2 = kp * kp;
  R px = r, py = r;
  for (uint64_t a = 0; a < 8; ++a) {
    uint64_t hp = orc_rng(c->seed, STREAM_RESET, (uint64_t)i, ep_id, 16u + 16u * (uint64_t)o + a);
    px = r + u24(hp) * (hx - r);
    py = r + u24b(hp) * (hy - r);
    R dsx = px - sx, dsy = py - sy, dgx = px - gx, dgy = py - gy;
    int ok = !occupied(m, map, (int64_t)FLOOR(px), (int64_t)FLOOR(py)) && FMA(dsx, dsx, dsy * dsy) > keep2 &&
             FMA(dgx, dgx, dgy * dgy) > keep2;
    if (ok) break;
  }
  uint64_t hv = orc_rng(c->seed, STREAM_RESET, (uint64_t)i, ep_id, 16u + 16u * (uint64_t)o + 8u);
  R pi = PI_R;
  R th = -pi + u24(hv) * (pi - (-pi));
  R lo = (R)c->dyn_speed_lo, hi = (R)c->dyn_speed_hi;
  R sp = lo + u24b(hv) * (hi - lo);
  R sn, cs;
  sincos_r(th, &sn, &cs);
  e->dyn[(4 * o + 0) * n + i] = px;
  e->dyn[(4 * o + 1) * n + i] = py;
  e->dyn[(4 * o + 2) * n + i] = sp * cs;
  e->dyn[(4 * o + 3) * n + i] = sp * sn;
}

/* One motion step of all of env i's obstacles (exported for the pins). */
void orc_dyn_advance(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i, R dt) {
  for (int32_t o = 0; o < c->n_dyn; ++o) dyn_move(c, m, e, i, o, dt);
}
int32_t orc_dyn_collide(const orc_config* c, const orc_envs* e, int32_t i, R x, R y) {
  return dyn_collide(c, e, i, x, y);
}

static R lerp_r(double lo, double hi, R u) {
  R l = (R)lo, hh = (R)hi;
  return l + u * (hh - l);
}

/* Episode start of env i (AutoReset and reset): every randomised parameter is
 * re-drawn from the counter RNG keyed by (seed, env, episode id), Sec. 3.2.4;
 * the robot starts near S with a random heading; velocities and the delay
 * queue are cleared. */
void orc_reset_env(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i, uint32_t ep_id, R* obs) {
  int32_t n = e->n_envs;
  uint64_t sd = c->seed;
  uint64_t h[8];
  for (int32_t s = 0; s < 8; ++s) h[s] = orc_rng(sd, STREAM_RESET, (uint64_t)i, ep_id, (uint64_t)s);
  e->f[F_DT * n + i] = lerp_r(c->dt_lo, c->dt_hi, u24(h[0]));
  uint32_t span = (uint32_t)(c->delay_hi - c->delay_lo + 1);
  e->b[B_DELAY * n + i] = (uint8_t)(c->delay_lo + (int32_t)((uint32_t)(h[1] >> 32) % span));
  e->f[F_K * n + i] = lerp_r(c->k_lo, c->k_hi, u24(h[2]));
  e->f[F_CAP * n + i] = lerp_r(c->cap_lo, c->cap_hi, u24(h[3]));
  e->f[F_SIGMA * n + i] = lerp_r(c->sigma_lo, c->sigma_hi, u24(h[4]));
  layout_t L = layout_of(c, m, e->env_map[i]);
  R jx = lerp_r(-c->start_jitter, c->start_jitter, u24(h[5]));
  R jy = lerp_r(-c->start_jitter, c->start_jitter, u24(h[6]));
  e->f[F_X * n + i] = L.sx + jx;
  e->f[F_Y * n + i] = L.sy + jy;
  R pi = PI_R;
  e->f[F_PHI * n + i] = -pi + u24(h[7]) * (pi - (-pi));
  e->f[F_VL * n + i] = (R)0;
  e->f[F_VA * n + i] = (R)0;
  e->u[U_STEP * n + i] = 0;
  e->u[U_EPID * n + i] = ep_id;
  e->b[B_Q0 * n + i] = NONE_ACTION;
  e->b[B_Q1 * n + i] = NONE_ACTION;
  for (int32_t o = 0; o < c->n_dyn; ++o) dyn_draw(c, m, e, i, ep_id, o, L.sx, L.sy, L.gx, L.gy);
  observe(c, m, e, i, obs);
}

void orc_reset(const orc_config* c, const orc_maps* m, orc_envs* e, R* obs) {
  int32_t stride = c->n_beams + 5;
  for (int32_t i = 0; i < e->n_envs; ++i) orc_reset_env(c, m, e, i, 0u, obs + (int64_t)i * stride);
}

/* One step of env i with action a.  Order: delay queue, target velocity,
 * Eq. 5, Eq. 6 (old heading), heading wrap, obstacle motion, collision,
 * LiDAR + noise, arrival / truncation, reward Eq. 11, observation,
 * AutoReset. */
static void step_env(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i, uint8_t a, R* obs,
                     R* rew, uint8_t* done, R* term_obs, uint32_t* status) {
  int32_t n = e->n_envs;
  int32_t B = c->n_beams;
  int32_t map = e->env_map[i];
  R* f = e->f;
  /* control delay: a FIFO of the last two actions; with delay d the
   * executed action is the one given d steps ago (none during the first d
   * steps of an episode, which targets zero velocity) */
  uint8_t d = e->b[B_DELAY * n + i];
  uint8_t q0 = e->b[B_Q0 * n + i], q1 = e->b[B_Q1 * n + i];
  uint8_t ahat = d == 0 ? a : (d == 1 ? q0 : q1);
  e->b[B_Q1 * n + i] = q0;
  e->b[B_Q0 * n + i] = a;
  if ((int32_t)a >= c->n_actions) *status |= 1u; /* invalid action index */
  R cap = f[F_CAP * n + i];
  R vhl = (R)0, vha = (R)0;
  if ((int32_t)ahat < c->n_actions) {
    vhl = (R)c->action_v[ahat] * cap;
    vha = (R)c->action_w[ahat] * cap;
  }
  /* Eq. 5 */
  R K = f[F_K * n + i];
  R omk = (R)1 - K;
  R vl = K * f[F_VL * n + i] + omk * vhl;
  R va = K * f[F_VA * n + i] + omk * vha;
  /* Eq. 6: new velocity, old heading */
  R phi = f[F_PHI * n + i], dt = f[F_DT * n + i];
  R s, co;
  sincos_r(phi, &s, &co);
  R x = f[F_X * n + i] - dt * (vl * co);
  R y = f[F_Y * n + i] - dt * (vl * s);
  phi = phi + dt * va;
  R pi = PI_R, twopi = (R)2 * PI_R;
  if (phi >= pi)
    phi = phi - twopi;
  else if (phi < -pi)
    phi = phi + twopi;
  f[F_X * n + i] = x;
  f[F_Y * n + i] = y;
  f[F_PHI * n + i] = phi;
  f[F_VL * n + i] = vl;
  f[F_VA * n + i] = va;
  uint32_t ep_step = e->u[U_STEP * n + i] + 1u;
  e->u[U_STEP * n + i] = ep_step;

  /* obstacles move with the env's control interval, then the collision
   * test sees the map and the moved discs */
  for (int32_t o = 0; o < c->n_dyn; ++o) dyn_move(c, m, e, i, o, dt);
  int32_t collide = orc_collide(c, m, map, x, y) || dyn_collide(c, e, i, x, y);
  obs_aux aux = observe(c, m, e, i, obs);
  R d1sq = FMA(aux.ddx, aux.ddx, aux.ddy * aux.ddy);
  R rg = (R)c->goal_radius;
  int32_t arrive = d1sq <= rg * rg;
  int32_t trunc = ep_step >= (uint32_t)c->t_max;
  /* Eq. 11 with the readings: r_d1 = 1 - d1/D, r_d2 = 1 - d2/(D/2) with d2 the
   * distance to the line S->G, r_v = [vl > v_max/2], r_alpha = 1 - |alpha|/pi,
   * r_d = -1 when the nearest noise-free range is below near_dist */
  layout_t L = layout_of(c, m, map);
  R d1 = SQRT(d1sq);
  R rd1 = (R)1 - d1 / L.D;
  R ex = L.gx - L.sx, ey = L.gy - L.sy;
  R px = x - L.sx, py = y - L.sy;
  R cr = ex * py - ey * px;
  R t2 = FABS(cr) / L.D / L.D;
  R rd2 = (R)1 - (t2 + t2);
  R vmax = (R)c->v_nom * cap;
  R rv = vl > (R)0.5 * vmax ? (R)1 : (R)0;
  R ra = (R)1 - FABS(aux.alpha) / pi;
  R rdn = aux.min_range < (R)c->near_dist ? (R)-1 : (R)0;
  R r = (R)0.3 * rd1;
  r = r + (R)0.1 * rd2;
  r = r + (R)0.3 * rv;
  r = r + (R)0.3 * ra;
  r = r + (R)0.1 * rdn;
  if (collide)
    r = (R)-10;
  else if (arrive)
    r = (R)75;
  *rew = r;
  uint8_t dn = (uint8_t)((collide ? 1 : 0) | (arrive ? 2 : 0) | (trunc ? 4 : 0));
  *done = dn;
  if (dn) {
    /* AutoReset: keep the true next observation, start a new episode */
    for (int32_t j = 0; j < B + 5; ++j) term_obs[j] = obs[j];
    orc_reset_env(c, m, e, i, e->u[U_EPID * n + i] + 1u, obs);
  }
}

void orc_step(const orc_config* c, const orc_maps* m, orc_envs* e, const uint8_t* act, R* obs, R* rew,
              uint8_t* done, R* term_obs, uint32_t* status) {
  int64_t stride = c->n_beams + 5;
  for (int32_t i = 0; i < e->n_envs; ++i)
    step_env(c, m, e, i, act[i], obs + i * stride, rew + i, done + i, term_obs + i * stride, status);
}

/* Step env i alone (the other envs are untouched); obs/term_obs are its
 * rows. */
void orc_step_one(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i, uint8_t a, R* obs, R* rew,
                  uint8_t* done, R* term_obs, uint32_t* status) {
  step_env(c, m, e, i, a, obs, rew, done, term_obs, status);
}

/* Network-free action source: uniform over the action table from the
 * counter RNG keyed by (seed, env, global step). */
uint8_t orc_random_action(const orc_config* c, int32_t i, uint64_t t) {
  uint64_t h = orc_rng(c->seed, STREAM_ACTION, (uint64_t)i, t, 0u);
  return (uint8_t)((uint32_t)(h >> 32) % (uint32_t)c->n_actions);
}

/* VEM exploration draw: a uniform in [0, 1) per (env, global step); the env
 * explores when it is below its exploration noise eps_i (Sec. 3.1.1). */
R orc_explore_uniform(const orc_config* c, int32_t i, uint64_t t) {
  return u24(orc_rng(c->seed, STREAM_ACTION, (uint64_t)i, t, 1u));
}

/* K steps of envs [i0, i1) alone with random actions from global step t0;
 * rewards and done flags are not kept (used to time the oracle). */
void orc_rollout_random_range(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t i0, int32_t i1,
                              int32_t K, uint64_t t0, uint32_t* status) {
  R obs[69], term[69], rew;
  uint8_t done;
  for (int32_t i = i0; i < i1; ++i)
    for (int32_t k = 0; k < K; ++k)
      step_env(c, m, e, i, orc_random_action(c, i, t0 + (uint64_t)k), obs, &rew, &done, term, status);
}

/* K steps with random actions starting at global step t0.  Per step k it
 * records the action, reward and done flags ([K][n] each); obs holds the
 * observation after the last step. */
void orc_rollout_random(const orc_config* c, const orc_maps* m, orc_envs* e, int32_t K, uint64_t t0, R* obs,
                        R* term_obs, uint8_t* act_seq, R* rew_seq, uint8_t* done_seq, uint32_t* status) {
  int32_t n = e->n_envs;
  for (int32_t k = 0; k < K; ++k) {
    uint8_t* act = act_seq + (int64_t)k * n;
    for (int32_t i = 0; i < n; ++i) act[i] = orc_random_action(c, i, t0 + (uint64_t)k);
    orc_step(c, m, e, act, obs, rew_seq + (int64_t)k * n, done_seq + (int64_t)k * n, term_obs, status);
  }
}
