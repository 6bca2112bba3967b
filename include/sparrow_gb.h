/*
 * sparrow_gb.h -- C ABI of the GB300 vectorized Sparrow environment step
 * (paper arxiv 2305.04180, "Color": Sec. 3.2 Sparrow simulator, Sec. 3.1
 * Actor-Sharer-Learner).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Return value: SG_OK (0) or a negative SG_E_* code.  No C++ exception
 *   crosses this boundary.  sg_strerror() names a code.
 * - "_dev" pointers are device pointers (cudaMalloc / torch tensors on the
 *   library's device), owned by the caller, contiguous, 16-byte aligned
 *   unless stated otherwise; the library never frees them.  Host pointers are
 *   plain host memory.  Handles (sg_sim_t, sg_qnet_t, sg_replay_t) own their
 *   device memory and release it in the matching _destroy call.
 * - Every call that takes an sg_stream_t enqueues its work on that stream
 *   (NULL = the legacy default stream) and returns without waiting; results
 *   are valid once the stream reaches that point.  Calls without a stream are
 *   synchronous.  Work on one handle must not run concurrently on two streams.
 * - Errors found on the device (a bad action index, a wait that ran out) are
 *   latched into a status word per handle; read it with sg_sim_status().
 * - Layouts: an observation row has obs_dim = n_beams + 5 floats:
 *   [0, n_beams)   LiDAR ranges / range_max (beams beyond an env's own beam
 *                  count read 1.0),
 *   n_beams + 0/1  goal vector in the robot frame (forward, left) / D,
 *   n_beams + 2    heading-to-goal angle alpha / pi,
 *   n_beams + 3/4  linear / angular velocity over their nominal maxima.
 *   Matrices are row-major [rows][cols].
 */
#ifndef SPARROW_GB_H
#define SPARROW_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sg_stream_t; /* same type as cudaStream_t */
typedef struct sg_sim* sg_sim_t;
typedef struct sg_qnet* sg_qnet_t;
typedef struct sg_replay* sg_replay_t;
typedef struct sg_graph* sg_graph_t;

enum {
  SG_OK = 0,
  SG_E_INVAL = -1,   /* a NULL handle/pointer, a size or enum out of range */
  SG_E_ALIGN = -2,   /* a device pointer without the documented alignment */
  SG_E_OOM = -3,     /* a device or host allocation failed */
  SG_E_CUDA = -4,    /* a CUDA runtime call failed */
  SG_E_DEVICE = -5,  /* the device status word holds an error */
  SG_E_TIMEOUT = -6  /* a bounded device-side wait ran out */
};

/* Device status bits (sg_sim_status). */
#define SG_DEV_BAD_ACTION 0x1u /* an action index >= n_actions was stepped */
#define SG_DEV_TIMEOUT 0x2u    /* a bounded spin-wait gave up */
#define SG_DEV_BOUNDS 0x4u     /* debug builds only: a computed map or ring index fell outside its
                                  array; the access was skipped (see sg_sim_status) */

/* Rollout action sources (sg_sim_rollout). */
#define SG_POLICY_RANDOM 0 /* uniform over the action table, counter RNG */
#define SG_POLICY_EPS_Q 1  /* VEM: eps_i-greedy over the Q-network */

/*
 * Simulation parameters (Sec. 3.2; nominal values in the paper's
 * simulation-parameter table).  Lengths are in cells (1 cell = 1 cm),
 * angles in radians, times in seconds.  Each *_lo/*_hi pair is the uniform
 * range that "vectorized diversity" (Sec. 3.2.4) re-draws per env at the start
 * of every episode; lo == hi fixes the value.
 */
typedef struct sg_sim_config {
  int32_t n_envs;      /* N >= 1 */
  int32_t n_beams;     /* B_max in [2, 64]; obs_dim = n_beams + 5 */
  int32_t n_actions;   /* in [1, 8] */
  int32_t t_max;       /* episode truncation length (steps), >= 1 */
  int32_t delay_lo;    /* control delay in steps, 0 <= lo <= hi <= 2 */
  int32_t delay_hi;
  float fov;           /* LiDAR fan, radians, in [0, 2 pi]; beam j at phi - fov/2 + j fov/(nb-1) */
  float range_max;     /* R_max, cells, > 0 */
  float march_step;    /* ray-march sample spacing, cells, > 0; R_max/step <= 4096 */
  float robot_radius;  /* collision disc radius, cells */
  float goal_radius;   /* arrival disc radius around the goal, cells */
  float near_dist;     /* reward term r_d = -1 when an obstacle is closer */
  float start_offset;  /* S = (off, off), G = (W - off, H - off) per map */
  float start_jitter;  /* start position jitter, uniform in +-jitter per axis */
  float dt_lo, dt_hi;        /* control interval */
  float k_lo, k_hi;          /* inertia factor K of Eq. 5 */
  float cap_lo, cap_hi;      /* velocity-range factor on the action table */
  float sigma_lo, sigma_hi;  /* LiDAR noise standard deviation, cells */
  float v_nom, w_nom;        /* nominal max linear / angular velocity */
  float action_v[8];         /* target linear velocity of each action */
  float action_w[8];         /* target angular velocity of each action */
  uint64_t seed;             /* counter-RNG key of every random draw */
  /*
   * Dynamic obstacles (optional; the paper's Sec. 5 names them as the
   * simulator's next capability, without a model).  n_dyn discs of radius
   * dyn_radius per env, re-drawn at every episode start: centre uniform over
   * [r, W - r] x [r, H - r] on a free cell farther than dyn_keepout from S and
   * G (first of up to 8 candidates), heading uniform, speed uniform in
   * [dyn_speed_lo, dyn_speed_hi] cells/s.  Each step, after the robot's
   * motion, a disc moves by dt * v; a centre leaving [r, W - r] (resp. H) is
   * mirrored back and that velocity component flips; a centre that would
   * enter an occupied cell stays and the velocity reverses.  The robot
   * collides when the centres are within robot_radius + dyn_radius; a LiDAR
   * sample inside a disc is a hit.  n_dyn = 0 (default): no obstacles, the
   * other fields are ignored.  Requires 2 r < every map side.  The SPLIT
   * rollout kernel does not support obstacles (sg_sim_set_launch rejects it).
   */
  int32_t n_dyn;             /* 0..8 */
  float dyn_radius;          /* > 0 when n_dyn > 0, cells */
  float dyn_speed_lo, dyn_speed_hi; /* 0 <= lo <= hi, cells / s */
  float dyn_keepout;         /* >= 0, cells */
  /*
   * Direction sectors of the march's acceleration structure (not part of the
   * step: hit indices are those of the plain march whatever the value).
   * 1: one skip map per map (Chebyshev clearance).  4, 8, 16 or 32: as many
   * "sector skip" planes per map in addition, each giving the number of
   * samples a ray of that direction sector can skip from a cell (about 2x
   * fewer march iterations at 16 on the benchmark maps); they cost
   * march_sectors bytes per map cell and are built at creation.  0: 16 when
   * the 16 planes of all maps fit in the GPU's L2 cache (126 MB on GB300:
   * 32 maps of 366 x 366 do), else 1.  Ignored (1) when march_step > 1,
   * where the march tests every sample.
   */
  int32_t march_sectors;
} sg_sim_config;

/* Read-only facts about a simulator (sg_sim_info). */
typedef struct sg_sim_info {
  int32_t n_envs;
  int32_t n_beams;
  int32_t obs_dim;
  int32_t n_maps;
  int64_t atlas_words;   /* 32-bit words of the bit-packed map atlas */
  int64_t state_bytes;   /* size of the sg_sim_get_state / set_state blob */
  int32_t device;        /* CUDA device ordinal the simulator lives on */
  int32_t march_sectors; /* sector planes per map in use (1: none) */
} sg_sim_info;

/* ---------------------------------------------------------------------- */
/* Simulator                                                               */
/* ---------------------------------------------------------------------- */

/*
 * Create N vectorized environments on the current CUDA device.
 * Sec. 3.2 (world matrix [x, y, phi, v_l, v_a, dt, K, O_xy], Sec. 3.2.3) and
 * Sec. 3.2 "Map customization": maps are binary occupancy grids.
 *   cfg        parameters (copied).
 *   n_maps     number of maps, >= 1.
 *   maps_host  n_maps host pointers; map m is a row-major uint8 grid of
 *              map_h[m] rows x map_w[m] columns, nonzero = occupied.  The
 *              library packs them into a device bit atlas (1 bit per cell,
 *              rows padded to 16 bytes) and does not keep the host pointers.
 *   map_w/h    map sides, each in [1, 16384].
 *   env_map    n_envs host ints: the map of each env, in [0, n_maps).
 *   env_beams  NULL (every env uses cfg->n_beams) or n_envs host ints in
 *              [2, cfg->n_beams]: per-env beam counts (uneven batching).
 *   out        receives the handle.
 * Synchronous.  Errors: SG_E_INVAL, SG_E_OOM, SG_E_CUDA.
 */
int sg_sim_create(const sg_sim_config* cfg, int32_t n_maps, const uint8_t* const* maps_host,
                  const int32_t* map_w, const int32_t* map_h, const int32_t* env_map,
                  const int32_t* env_beams, sg_sim_t* out);

/* Release every device buffer of the simulator.  Synchronous. */
int sg_sim_destroy(sg_sim_t sim);

/* Static facts (sizes) of a simulator. */
int sg_sim_info_get(sg_sim_t sim, sg_sim_info* info);

/*
 * Start episode 0 of every env (Sec. 3.2.4: every randomised parameter is
 * drawn per env; the robot starts near S with a random heading) and write the
 * first observation.
 *   seed     replaces cfg->seed for this and every later draw.
 *   obs_dev  N x obs_dim floats (may be NULL: no observation written).
 */
int sg_sim_reset(sg_sim_t sim, uint64_t seed, float* obs_dev, sg_stream_t stream);

/*
 * One vectorized step of every env (Sec. 3.2: Eq. 5 and Eq. 6 kinematics with
 * control delay, LiDAR ray casting with sensor noise, collision, arrival,
 * reward Eq. 11 of Sec. 4.3.1, and AutoReset of done envs, Sec. 3.2.5).
 *   act_dev       N uint8 action indices; an index >= n_actions counts as
 *                 "no command" (zero target velocity) and sets
 *                 SG_DEV_BAD_ACTION in the status word.
 *   obs_dev       N x obs_dim floats: observation after the step (after the
 *                 reset for done envs).
 *   rew_dev       N floats.
 *   done_dev      N uint8: bit0 collided, bit1 arrived, bit2 truncated.
 *   term_obs_dev  N x obs_dim floats or NULL: for done envs the observation
 *                 before the reset (rows of other envs are not written).
 * No alignment beyond 4 bytes is required of these buffers.
 */
int sg_sim_step(sg_sim_t sim, const uint8_t* act_dev, float* obs_dev, float* rew_dev, uint8_t* done_dev,
                float* term_obs_dev, sg_stream_t stream);

/*
 * K vectorized steps in one persistent launch (Alg. 1 steps 2-5 of the
 * paper's Actor, the "vectorized data collection").  Each step picks the
 * actions on the device:
 *   SG_POLICY_RANDOM  uniform over the action table from the counter RNG;
 *   SG_POLICY_EPS_Q   VEM (Sec. 3.1.1): with probability eps_dev[i] the random
 *                     action, otherwise argmax_a Q(s, a) of `qnet` (lowest
 *                     index on ties), Q evaluated in BF16 with FP32
 *                     accumulation inside the same kernel.
 *   qnet          required for SG_POLICY_EPS_Q, ignored otherwise.
 *   eps_dev       N floats (required for SG_POLICY_EPS_Q).
 *   replay        NULL or a ring that receives one transition per env-step
 *                 (s, a, r, s', terminal), Alg. 1 step 5.
 *   obs_dev       NULL or N x obs_dim floats: observation after the last step.
 *   obs_seq_dev   NULL or K x N x obs_dim floats: observation after each step
 *                 (after the reset for envs that were done).
 *   act_seq_dev   NULL or K x N uint8: action taken at each step.
 *   rew_seq_dev   NULL or K x N floats.
 *   done_seq_dev  NULL or K x N uint8 (flags as in sg_sim_step).
 * K in [1, 1 << 20].
 */
int sg_sim_rollout(sg_sim_t sim, int32_t K, int32_t policy, sg_qnet_t qnet, const float* eps_dev,
                   sg_replay_t replay, float* obs_dev, float* obs_seq_dev, uint8_t* act_seq_dev,
                   float* rew_seq_dev, uint8_t* done_seq_dev, sg_stream_t stream);

/*
 * Launch configuration of the network-free rollout (uneven batching and the
 * autotuner).  Results never depend on it: every kernel computes the same
 * float32 step.  kernel:
 *   SG_ROLLOUT_GRID   one warp per env, warps_per_block envs per CTA
 *                     (1, 2, 4 (default), 8, 16).
 *   SG_ROLLOUT_QUEUE  a persistent grid of warps_per_block-warp CTAs
 *                     (blocks_per_sm per SM, 0 = the occupancy limit) pulls
 *                     envs from a work list through a device counter; order
 *                     0 = index order, 1 = sorted by cost (beams x map size),
 *                     longest first.
 *   SG_ROLLOUT_SPLIT  warps_per_env (1..8) warps share one env: with random
 *                     actions the pose chain (motion, collision, arrival,
 *                     AutoReset draws) never depends on the LiDAR, so every
 *                     warp replays it and warp w computes the scans,
 *                     observations and rewards of the steps i = w (mod W);
 *                     max(1, warps_per_block / W) envs per CTA,
 *                     warps_per_block 1..8.
 *   SG_ROLLOUT_PIPE   per env one warp computes the pose chain of 32-step
 *                     chunks into shared memory (motion run ahead through
 *                     the chunk, the chunk's steps tested together, restart
 *                     after each episode end) and then joins obs_warps
 *                     (1..15) warps that compute the scans, observations and
 *                     rewards of the previous chunk, taking steps from a
 *                     shared counter; min(3, max(1, warps_per_block /
 *                     (1 + obs_warps))) envs per CTA, warps_per_block 1..16;
 *                     order 0 = index order, 1 = envs grouped by map (CTAs
 *                     share maps, so fewer maps compete for each SM's L1).
 *                     segment > 0 (a multiple of 32, at most 1 << 20) slices
 *                     the rollout in time: a resident grid takes (segment,
 *                     CTA's envs) items in order, each after the previous
 *                     segment of its envs is stored, so that no CTA slot
 *                     idles in a last partial wave; segment 0 (default) runs
 *                     every env's K steps in one CTA.  The waits are
 *                     bounded (wait_iters sleeps of ~256 ns each; 0 = the
 *                     default 2^22, about a second): on timeout the status
 *                     word gets SG_DEV_TIMEOUT, the other CTAs stop at
 *                     their next item, and the outputs and env state of
 *                     that launch are incomplete.
 * Synchronous (computes and uploads the work list on first use).
 */
#define SG_ROLLOUT_GRID 0
#define SG_ROLLOUT_QUEUE 1
#define SG_ROLLOUT_SPLIT 2
#define SG_ROLLOUT_PIPE 3
typedef struct sg_launch {
  int32_t kernel;
  int32_t warps_per_block;
  int32_t warps_per_env;
  int32_t obs_warps;
  int32_t blocks_per_sm;
  int32_t order;
  int32_t segment;     /* SG_ROLLOUT_PIPE time slicing, steps; 0 = none */
  int32_t wait_iters;  /* bound of a time-sliced item's wait; 0 = default */
} sg_launch;
int sg_sim_set_launch(sg_sim_t sim, const sg_launch* cfg);
int sg_sim_get_launch(sg_sim_t sim, sg_launch* cfg);

/*
 * Copy the complete env state to / from host memory (checkpoint / resume;
 * every random draw is keyed by state, so a restored run continues
 * bit-identically).  Blob layout, N = n_envs:
 *   float    [9][N]  x, y, phi, v_l, v_a, dt, K, cap, sigma
 *   uint32_t [3][N]  ep_step, ep_id, t (steps since reset)
 *   uint32_t [1][N]  fifo: last action | previous action << 8 | delay << 16
 *                    (255 = no action yet)
 *   float    [4 n_dyn][N]  dynamic obstacles (only when n_dyn > 0): obstacle
 *                    o at rows 4o..4o+3 = centre x, y, velocity vx, vy
 * *bytes: in = size of host_buf, out = bytes used (info.state_bytes).
 * Synchronous.
 */
int sg_sim_get_state(sg_sim_t sim, void* host_buf, size_t* bytes);
int sg_sim_set_state(sg_sim_t sim, const void* host_buf, size_t bytes);
/*
 * sg_sim_set_state ordered on `stream` instead of synchronous: the upload
 * (the same blob, bytes = info.state_bytes, else SG_E_INVAL) runs after the
 * work enqueued on the stream before it, so a caller can queue the next
 * rollout's start state behind the current one.  host_buf must stay valid
 * and unchanged until the copy has run; page-locked memory makes the copy
 * asynchronous (with pageable memory the call returns once the data is
 * staged).
 */
int sg_sim_set_state_async(sg_sim_t sim, const void* host_buf, size_t bytes, sg_stream_t stream);

/*
 * Copy the bit-packed map atlas to the host: for map m, row cy starts at
 * word offs_host[m] + cy * row_words_host[m]; bit (cx & 31) of word
 * (cx >> 5) of that row is cell cx.  Any of the three outputs may be NULL.
 * *words: in = capacity of atlas_host in words, out = atlas words.
 * Synchronous.
 */
int sg_sim_get_atlas(sg_sim_t sim, uint32_t* atlas_host, size_t* words, int64_t* offs_host,
                     int32_t* row_words_host);

/*
 * Copy the skip maps to the host (the acceleration structure of the ray
 * march, not part of the paper's step): for map m, byte offs_host[m] +
 * cy * W + cx is 0 on occupied cells and max(1, c - 1) on free cells, where
 * c = min(255, Chebyshev distance in cells from cell (cx, cy) to the nearest
 * occupied cell), cells outside the map counting as occupied (the number of
 * march samples that can be skipped from there).  *bytes: in = capacity of
 * host, out = total bytes (sum of W x H).  host and offs_host may be NULL.
 * Synchronous.
 */
int sg_sim_get_clearance(sg_sim_t sim, uint8_t* host, size_t* bytes, int64_t* offs_host);

/*
 * Copy the sector skip planes to the host (see march_sectors in
 * sg_sim_config; an acceleration structure, not part of the paper's step).
 * Plane s of map m: byte offs_host[m] + s * W * H + cy * W + cx, for the ray
 * directions whose angle lies in [-pi + s 2pi/S, -pi + (s+1) 2pi/S), S =
 * march_sectors: 0 on occupied cells, else a number of march samples J >= 1
 * such that from a sample in cell (cx, cy) the next J - 1 samples of such a
 * ray lie in free cells of the map.  *bytes: in = capacity of host, out =
 * total bytes (S x sum of W x H; 0 when S = 1).  host and offs_host may be
 * NULL.  Synchronous.
 */
int sg_sim_get_sector_skip(sg_sim_t sim, uint8_t* host, size_t* bytes, int64_t* offs_host);

/*
 * Read (synchronously) and clear the device status word: SG_DEV_* bits.
 * Returns SG_E_DEVICE if any bit was set, SG_OK otherwise.  In the debug
 * build (libsparrowgb_debug.so, compiled with SG_DEBUG_BOUNDS) every skip-map
 * load of the ray march, every bit-row load of the collision test and every
 * ring entry the learner samples is checked against its array first; an
 * index outside it skips the access (the march then reports a hit there) and
 * sets SG_DEV_BOUNDS, which this call also reports and clears (for every
 * simulator and network of the process).  The regular build has no checks.
 */
int sg_sim_status(sg_sim_t sim, uint32_t* device_status);

/* ---------------------------------------------------------------------- */
/* Learned part: Q-networks, replay ring, TD learner                        */
/* ---------------------------------------------------------------------- */

/*
 * Q-network of one of two architectures, ReLU between layers, 5 discrete
 * actions (Sec. 4.3.1):
 *   SG_QNET_DUELING  in -> 256 -> 256 -> (1 value + 5 advantages),
 *                    Q = V + A - mean(A) (the dueling architecture the paper
 *                    cites in Sec. 2).  Flat parameter order (set/get):
 *                    W1[256][n_in], b1[256], W2[256][256], b2[256], W3[6][256],
 *                    b3[6]; row 0 of W3/b3 is the value head.
 *   SG_QNET_PAPER    the paper's four fully connected layers [32, 256, 128, 5]
 *                    of the Task2Task experiment (Sec. 4.3.2): in -> 256 ->
 *                    128 -> 5, the outputs are the Q-values.  Flat order
 *                    W1[256][n_in], b1[256], W2[128][256], b2[128], W3[5][128],
 *                    b3[5].
 * Inference and learning run on the tensor cores with BF16 weights and
 * activations and FP32 accumulation; FP32 master weights, a target copy and
 * Adam moments stay on the device.
 *   n_in       input width = the simulator's obs_dim, in [1, 69].
 *   arch       SG_QNET_DUELING or SG_QNET_PAPER (else SG_E_INVAL).
 *   max_batch  largest sg_td_train_step batch, in [1, 65536] (sizes the
 *              learner's scratch buffers).
 *   seed       parameters start uniform in +-1/sqrt(fan_in), parameter j of
 *              the flat order drawn from the counter RNG with this seed; the
 *              target copy equals them.
 * Synchronous.
 */
#define SG_QNET_DUELING 0
#define SG_QNET_PAPER 1
int sg_qnet_create(int32_t n_in, int32_t arch, int32_t max_batch, uint64_t seed, sg_qnet_t* out);
int sg_qnet_destroy(sg_qnet_t q);
/* Number of parameters of the network's flat order (77,062 for the dueling
 * network at n_in = 37, 41,989 for the paper's at n_in = 32). */
int sg_qnet_num_params(sg_qnet_t q, int64_t* n);
/* Copy parameters from / to host floats; which: 0 online, 1 target, 2 both
 * (set only).  Setting rebuilds the BF16 copies.  Synchronous. */
int sg_qnet_set_params(sg_qnet_t q, const float* host, int64_t n, int32_t which);
int sg_qnet_get_params(sg_qnet_t q, float* host, int64_t n, int32_t which);
/* Adam first / second moments (either pointer may be NULL) and the number of
 * optimiser steps taken.  Synchronous. */
int sg_qnet_get_optimizer(sg_qnet_t q, float* m_host, float* v_host, int64_t n, uint64_t* steps);
/* Restore the Adam moments and the optimiser step count (checkpoint
 * resume; with the parameters and the ring restored too, training continues
 * bit-identically).  Synchronous. */
int sg_qnet_set_optimizer(sg_qnet_t q, const float* m_host, const float* v_host, int64_t n, uint64_t steps);

/*
 * Envs per CTA of the fused rollout: 16 or 32 (one warp each, the network on
 * mma.sync tiles; the network's BF16 weights take most of an SM's shared
 * memory, so one CTA runs per SM), 128 (the tcgen05 kernel: 4 envs per warp,
 * the network as one 128-row tile on the fifth-generation tensor cores), or
 * 0 (default): 128 when the envs fill every SM with 128-env CTAs and there
 * are no moving obstacles, else 32 when that needs fewer waves than 16.
 * The simulator values do not depend on it; the Q values of the tcgen05
 * kernel differ in the FP32 summation order only (so greedy actions can
 * differ where two actions' Q values are within that rounding).
 */
int sg_qnet_set_rollout_rows(sg_qnet_t q, int32_t rows);

/*
 * At most rollout_ctas CTAs (one per SM) for the tcgen05 fused rollout run
 * with this network, and at most learner_ctas for its tcgen05 TD step (0 =
 * every SM, the default; negative: SG_E_INVAL).  The ASL framework runs the
 * actor and the learner in parallel (Sec. 3.1, Alg. 1 and 2): a rollout and
 * a learning step launched on concurrent streams (or graph branches) with
 * caps that add up to the SM count each keep SMs of their own instead of
 * taking turns.  Results do not depend on the caps (the rollout's items and
 * the learner's jobs are taken from device counters by whichever CTAs run).
 */
int sg_qnet_set_grid_limit(sg_qnet_t q, int32_t rollout_ctas, int32_t learner_ctas);

/*
 * Model upload (Alg. 2 step 3 / Alg. 1 step 1: the actor takes the learner's
 * latest parameters every U optimisation steps): dst's online network takes
 * src's online parameters and BF16 copy, stream-ordered.  Same n_in.
 */
int sg_qnet_copy_params(sg_qnet_t dst, sg_qnet_t src, sg_stream_t stream);

/*
 * Batched inference: q_dev[M][5] = Q(obs_dev[M][n_in]) with the online
 * network, on the fifth-generation tensor cores (tcgen05: persistent CTAs
 * over 128-row tiles, BF16 weights and inputs in shared memory, FP32
 * accumulators and the BF16 hidden activations in tensor memory; the same
 * BF16 recipe as the fused rollout).  obs_dev and q_dev are device
 * pointers, M >= 1; SG_E_INVAL for a null handle or pointer.  If a
 * device-side wait runs out (it should not), the rows of that CTA are NaN.
 */
int sg_qnet_forward(sg_qnet_t q, const float* obs_dev, int32_t M, float* q_dev, sg_stream_t stream);

/*
 * Device replay ring (Alg. 1 step 5 adds one batch of N transitions per
 * vectorized step; Alg. 2 step 1 samples a mini-batch).  Entry
 * e = slot * n_envs + env, slot = (step index) mod slots_per_env; capacity =
 * slots_per_env * n_envs transitions of (s, a, r, s', terminal) with s, s'
 * float[obs_dim], terminal = collided or arrived.  The learner samples only
 * the min(steps, slots_per_env - reserve_slots) most recently completed
 * slots: with reserve_slots >= the longest rollout that may run concurrently
 * with a training step (on another stream), no sample can be a slot that
 * rollout is still writing.  0 <= reserve_slots < slots_per_env.
 * Synchronous.
 */
int sg_replay_create(int32_t slots_per_env, int32_t n_envs, int32_t obs_dim, int32_t reserve_slots,
                     sg_replay_t* out);
int sg_replay_destroy(sg_replay_t r);
/* Capacity, vectorized steps recorded so far (synchronous read) and the
 * device arrays (s, s2: [cap][obs_dim] float; a, term: [cap] uint8;
 * r: [cap] float).  Any output may be NULL. */
int sg_replay_info(sg_replay_t r, int64_t* capacity, uint64_t* steps_recorded, void** s_dev, void** s2_dev,
                   void** a_dev, void** r_dev, void** term_dev);

/* Copy ring entries [first, first + count) to host arrays (any may be NULL).
 * Synchronous. */
int sg_replay_read(sg_replay_t r, int64_t first, int64_t count, float* s_host, float* s2_host, uint8_t* a_host,
                   float* r_host, uint8_t* term_host);
/* Write ring entries [first, first + count) from host arrays (all five
 * required when count > 0) and set the recorded-step counter (checkpoint
 * resume).  Synchronous. */
int sg_replay_write(sg_replay_t r, int64_t first, int64_t count, const float* s_host, const float* s2_host,
                    const uint8_t* a_host, const float* r_host, const uint8_t* term_host, uint64_t steps_recorded);

/*
 * One optimisation step of the learner (Alg. 2 steps 1-2 with DDQN): sample
 * `batch` ring entries uniformly from the completed slots (see
 * sg_replay_create; counter RNG keyed by seed and the optimiser step count), y = r + gamma (1 - terminal)
 * Q_target(s', argmax_a Q_online(s', a)), loss = mean Huber(Q(s, a) - y)
 * (delta 1), gradient by backpropagation, Adam (beta 0.9 / 0.999, eps 1e-8)
 * with learning rate lr; when the step count reaches a multiple of
 * target_every (> 0) the target network takes the online weights.
 *   lr = 0      computes loss and gradient only (no update, step count kept).
 *   loss_dev    NULL or 1 float: the batch loss.
 *   grad_dev    NULL or num_params floats: the summed gradient.
 * The replay's obs_dim must equal n_in; batch in [1, max_batch].
 * Device-side failure: when a weight-image copy into shared memory does not
 * complete within its bounded wait, or a sampled transition's action is not
 * below 5 (possible only for entries written by sg_replay_write), the step
 * makes no update: loss_dev and every grad_dev entry are NaN, and the
 * parameters, the target copy, the Adam moments and the step count stay as
 * they were.  The return code is SG_OK (the failure is found on the device,
 * after the call returned); check loss_dev for NaN.
 */
int sg_td_train_step(sg_qnet_t q, sg_replay_t replay, int32_t batch, float gamma, float lr, int32_t target_every,
                     uint64_t seed, float* loss_dev, float* grad_dev, sg_stream_t stream);

/*
 * VEM exploration noise (Sec. 3.1.1, "Vectorized data collection"; schedule
 * values of the hyper-parameter table): writes eps_dev[i] for the sim's n
 * envs at the current number of interacting steps T = n * t, where t is env
 * 0's step counter on the device (so a captured graph advances the schedule
 * as it replays).  The exploring interval
 *     OR(T) = or_start + (or_final - or_start) * min(1, T / decay_steps)
 * (a real number of envs) takes the last envs of the index range: env i with
 * i >= n - OR gets e_min + e_max * (i - (n - OR)) / (OR - 1), the others (the
 * exploiting interval) get e_min.  With OR = n this is e_min for env 0 up to
 * e_min + e_max for env n - 1.  Evaluated in float64, stored as float.
 *   2 <= or_final <= n, 2 <= or_start <= n, decay_steps > 0, e_min, e_max >= 0.
 * eps_dev: n floats, caller-owned device memory.  Asynchronous on stream.
 */
int sg_vem_eps(sg_sim_t sim, float e_min, float e_max, double or_start, double or_final, double decay_steps,
               float* eps_dev, sg_stream_t stream);

/*
 * TD loss and gradient that allocates nothing (the paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * code under a fixed memory budget, inside another framework's allocator, or
 * where cudaMalloc is not allowed -- and so cannot create an sg_qnet_t).
 * Computes what sg_td_train_step computes with lr = 0, for an explicit batch
 * instead of ring samples: y_i = r_i + gamma (1 - term_i)
 * Q_target(s2_i, argmax_a Q(s2_i, a)), loss = mean Huber(Q(s_i, a_i) - y_i),
 * and its gradient w.r.t. the online parameters.
 *   params_dev, target_params_dev  flat FP32 parameters (the dueling
 *                 network's order of sg_qnet_set_params) of the online and the
 *                 target network.
 *   n_in          input width, in [1, 69].
 *   s_dev, s2_dev batch x n_in floats; a_dev, term_dev batch uint8 (a < 5);
 *                 r_dev batch floats.  All caller-owned device memory.
 *   batch         in [1, 256].
 *   loss_dev      NULL or 1 float; grad_dev num_params floats (outputs).
 * An action index of 5 or more in a_dev, or a weight-image copy that does
 * not complete within its bounded wait, makes the whole result NaN (loss_dev
 * and every grad_dev entry), never a partial or a previous call's gradient.
 * Scratch: one file-scope device array of about 5.8 MB (BF16 weight images,
 * targets, per-CTA partial gradients, a failure word) that every GPU loading
 * the library holds until the process exits.  Every call shares it, clears
 * its failure word and overwrites all of it that it reads, so nothing
 * carries over between calls; calls that
 * overlap on the GPU (two streams, two threads) race on it and must be
 * serialised by the caller.  The first call on a device looks up the array's
 * device address and sets kernel attributes (no allocation); make that first
 * call before any stream capture.  Sizes beyond the limits return
 * SG_E_INVAL with a message in sg_last_cuda_error().  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 */
int sg_td_grad_noalloc(const float* params_dev, const float* target_params_dev, int32_t n_in, const float* s_dev,
                       const uint8_t* a_dev, const float* r_dev, const float* s2_dev, const uint8_t* term_dev,
                       int32_t batch, float gamma, float* loss_dev, float* grad_dev, sg_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Measurement                                                             */
/* ---------------------------------------------------------------------- */

/*
 * Read-bandwidth probe (not part of the paper's method: the measured
 * denominator of the L2 roofline reported for the simulator kernels).
 * `reps` passes of 16-byte loads cached in L2 only (ld.global.cg) over
 * buf_dev[0, bytes), by a grid of every 512-thread CTA that fits the GPU at
 * once (4 per SM); a buffer smaller than L2 is read from L2 after the first
 * pass, so bytes x reps / time is the L2 read bandwidth.  Each CTA XORs
 * what it read into sink_dev[its index] (so the loads cannot be dropped);
 * sink_words must be >= the grid (4 x the SM count suffices).
 * bytes: a multiple of 16, >= 16; buf_dev 16-byte aligned; reps >= 1; else
 * SG_E_INVAL.  Caller-owned device memory.  Asynchronous on stream.
 */
int sg_probe_read(const void* buf_dev, size_t bytes, int32_t reps, uint32_t* sink_dev, int32_t sink_words,
                  sg_stream_t stream);

/* ---------------------------------------------------------------------- */
/* CUDA graphs of rollouts and learner steps                                */
/* ---------------------------------------------------------------------- */

/*
 * Capture the library calls enqueued on `stream` between sg_graph_begin and
 * sg_graph_end (thread-local capture mode) into an executable graph; replay
 * it with sg_graph_launch.  Every counter the kernels use (per-env step
 * counts, the ring position, the optimiser step) lives on the device, so a
 * replay continues from where the previous one stopped: capturing K-step
 * rollouts once and replaying them equals calling them again.  Buffers
 * passed to the captured calls must stay valid while the graph exists.
 * Other streams may join the capture through events recorded on `stream`
 * and must rejoin it before sg_graph_end.  `stream` must not be NULL.
 */
int sg_graph_begin(sg_stream_t stream);
int sg_graph_end(sg_stream_t stream, sg_graph_t* out);
int sg_graph_launch(sg_graph_t g, sg_stream_t stream);
int sg_graph_num_nodes(sg_graph_t g, int64_t* n);
int sg_graph_destroy(sg_graph_t g);

/* Human-readable name of an SG_* return code. */
const char* sg_strerror(int code);

/* Text of the last CUDA error seen by this thread inside the library. */
const char* sg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SPARROW_GB_H */
