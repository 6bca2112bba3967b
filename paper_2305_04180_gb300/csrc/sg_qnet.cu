// sg_qnet.cu -- the learned part: dueling Q-network (Sec. 2 "Dueling DQN",
// Sec. 4.3.1 discrete actions), the VEM eps-greedy rollout with the network
// fused into the simulator loop (Sec. 3.1.1, Alg. 1), the device replay ring
// (Alg. 1 step 5, Alg. 2 step 1) and the double-DQN learner with Adam
// (Alg. 2 step 2; appendix hyperparameter table).
//
// Networks (SG_QNET_DUELING): in -> 256 -> 256 -> 6 (value + 5 advantages),
// ReLU, Q = V + A - mean(A); (SG_QNET_PAPER) the paper's in -> 256 -> 128 ->
// 5 with Q the outputs (Sec. 4.3.2).  The kernels run both at the dueling
// shapes: the paper network's 128 second-layer units and 5 outputs sit in
// the first rows of the 256-unit / 6-output storage and every other weight
// and bias stays exactly zero (its pre-activation is 0, so the ReLU mask
// zeroes its gradient and Adam never moves it, and adding its zero products
// leaves the other sums unchanged); only the head differs.  Weights are BF16
// on the tensor cores with FP32 accumulation; FP32 master weights, Adam
// moments and a target copy live on the device.  Flat parameter order inside
// (padded): W1[256][in] b1[256] W2[256][256] b2[256] W3[6][256] b3[6]; the
// C ABI shows each network's own (compact) order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sg_device.cuh"
#include "sg_host.h"
#include "sg_mma.cuh"
#include "sg_tc.cuh"
#include "sparrow_gb.h"

using namespace sg;

namespace {

constexpr int kHid = 256;
constexpr int kLdh = kHid + 8;  // padded row of a 256-wide BF16 matrix
constexpr int kOut = 6;
constexpr int kOutPad = 8;
constexpr int kTile = 16;       // envs / samples per CTA = warps per CTA
constexpr int kThreads = kTile * 32;
constexpr uint32_t kStreamSample = 4;
constexpr uint32_t kStreamInit = 5;

// Byte layout of the BF16 weight image (identical in global and shared memory).
struct ImgLayout {
  int n_in, k1, ld1;   // input width, padded to 16, row stride
  int w1, w2, w3, b1, b2, b3, bytes;
  int plain;           // 1: the outputs are the Q-values (the paper's network)
};

ImgLayout img_layout(int n_in, int plain = 0) {
  ImgLayout L;
  L.n_in = n_in;
  L.plain = plain;
  L.k1 = (n_in + 15) / 16 * 16;
  L.ld1 = L.k1 + 8;
  L.w1 = 0;
  L.w2 = L.w1 + kHid * L.ld1 * 2;
  L.w3 = L.w2 + kHid * kLdh * 2;
  L.b1 = L.w3 + kOutPad * kLdh * 2;
  L.b2 = L.b1 + kHid * 4;
  L.b3 = L.b2 + kHid * 4;
  L.bytes = (L.b3 + kOutPad * 4 + 15) / 16 * 16;
  return L;
}

// Offsets of the flat FP32 parameter vector.
struct ParamLayout {
  int w1, b1, w2, b2, w3, b3, total;
};
// Floats per CTA row of the gradient partials: every parameter, the Huber
// sum, padded to a multiple of 4 so that rows start 16-byte aligned.
__host__ __device__ constexpr long long partial_stride(int total) { return (total + 1 + 3) / 4 * 4; }

ParamLayout param_layout(int n_in) {
  ParamLayout P;
  P.w1 = 0;
  P.b1 = P.w1 + kHid * n_in;
  P.w2 = P.b1 + kHid;
  P.b2 = P.w2 + kHid * kHid;
  P.w3 = P.b2 + kHid;
  P.b3 = P.w3 + kOut * kHid;
  P.total = P.b3 + kOut;
  return P;
}

// The paper network's compact parameter index of padded index i, or -1 for a
// padding entry (always zero): W1[256][in] b1[256] W2[128][256] b2[128]
// W3[5][128] b3[5].
constexpr int kPaperH2 = 128;
__host__ __device__ inline int paper_index(int i, const ParamLayout& P, int n_in) {
  if (i < P.w2) return i;  // W1, b1 unchanged
  const int c_w2 = P.w2, c_b2 = c_w2 + kPaperH2 * kHid, c_w3 = c_b2 + kPaperH2, c_b3 = c_w3 + 5 * kPaperH2;
  if (i < P.b2) {
    const int j = i - P.w2, r = j / kHid, k = j % kHid;
    return r < kPaperH2 ? c_w2 + r * kHid + k : -1;
  }
  if (i < P.w3) {
    const int r = i - P.b2;
    return r < kPaperH2 ? c_b2 + r : -1;
  }
  if (i < P.b3) {
    const int j = i - P.w3, o = j / kHid, k = j % kHid;
    return o < 5 && k < kPaperH2 ? c_w3 + o * kPaperH2 + k : -1;
  }
  const int o = i - P.b3;
  return o < 5 ? c_b3 + o : -1;
}
inline int paper_params(int n_in) { return kHid * n_in + kHid + kPaperH2 * kHid + kPaperH2 + 5 * kPaperH2 + 5; }

}  // namespace

// Device view of a replay ring: slot-major SoA, entry e = slot * n_envs + env.
struct ReplayDev {
  float* s;              // [cap][obs_dim]
  float* s2;             // [cap][obs_dim]
  uint8_t* a;            // [cap]
  float* r;              // [cap]
  uint8_t* term;         // [cap] collided or arrived
  unsigned long long* steps;  // vectorized steps recorded so far
  int slots, n_envs, obs_dim;
  int reserve;           // newest slots the learner never samples (an actor may be writing them)
};

struct sg_replay {
  ReplayDev d;
  long long cap = 0;
  int device = 0;
};

struct sg_qnet {
  int n_in = 0;
  int arch = SG_QNET_DUELING;
  int device = 0;
  ImgLayout IL;
  ParamLayout PL;
  float* master = nullptr;  // [P]
  float* target = nullptr;  // [P]
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  uint8_t* img = nullptr;    // online BF16 image
  uint8_t* img_t = nullptr;  // target BF16 image
  unsigned long long* step = nullptr;  // optimiser steps taken (device)
  unsigned* td_fail = nullptr;         // SG_TD_FAIL_* bits of the current TD step (device), cleared per step
  // learner scratch, sized for max_batch
  int max_batch = 0;
  float* partial = nullptr;  // [max_batch / kTile][P + 1] (last entry: loss)
  float* y = nullptr;        // [max_batch] TD targets
  int* idx = nullptr;        // [max_batch] sampled ring entries
  int rollout_mt = 0;        // m-tiles per CTA of the fused rollout (0 = choose by waves)
  int lim_rollout = 0;       // CTA caps of the tcgen05 rollout / learner grids (0 = every SM)
  int lim_learner = 0;
  uint8_t* img_tc = nullptr; // the online weights in the tensor cores' shared-memory layout (batched forward)
  uint8_t* img_tc_t = nullptr; // the target weights in the same layout (tcgen05 learner)
  float* q2 = nullptr;       // [2][max_batch][5] Q-values of the sampled next states (tcgen05 learner)
  unsigned* td_sync = nullptr;  // [1 + max_batch / 128] job counter and per-tile counters (tcgen05 learner)
  int sms = 0;               // multiprocessors of the device (persistent grids)
};

// --------------------------------------------------------------- kernels

// Image entries from the FP32 parameters: W1/W2/W3 rounded to BF16 into the
// padded layout (pad entries zero), biases copied.
__global__ void k_build_image(const float* __restrict__ th, uint8_t* __restrict__ img, ImgLayout L, ParamLayout P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  bf16* W1 = reinterpret_cast<bf16*>(img + L.w1);
  bf16* W2 = reinterpret_cast<bf16*>(img + L.w2);
  bf16* W3 = reinterpret_cast<bf16*>(img + L.w3);
  float* b1 = reinterpret_cast<float*>(img + L.b1);
  float* b2 = reinterpret_cast<float*>(img + L.b2);
  float* b3 = reinterpret_cast<float*>(img + L.b3);
  const int n1 = kHid * L.ld1, n2 = kHid * kLdh, n3 = kOutPad * kLdh;
  if (i < n1) {
    const int r = i / L.ld1, k = i % L.ld1;
    W1[i] = __float2bfloat16_rn(k < L.n_in ? th[P.w1 + r * L.n_in + k] : 0.0f);
  } else if (i < n1 + n2) {
    const int j = i - n1, r = j / kLdh, k = j % kLdh;
    W2[j] = __float2bfloat16_rn(k < kHid ? th[P.w2 + r * kHid + k] : 0.0f);
  } else if (i < n1 + n2 + n3) {
    const int j = i - n1 - n2, r = j / kLdh, k = j % kLdh;
    W3[j] = __float2bfloat16_rn(r < kOut && k < kHid ? th[P.w3 + r * kHid + k] : 0.0f);
  } else if (i < n1 + n2 + n3 + kHid) {
    const int j = i - n1 - n2 - n3;
    b1[j] = th[P.b1 + j];
  } else if (i < n1 + n2 + n3 + 2 * kHid) {
    const int j = i - n1 - n2 - n3 - kHid;
    b2[j] = th[P.b2 + j];
  } else if (i < n1 + n2 + n3 + 2 * kHid + kOutPad) {
    const int j = i - n1 - n2 - n3 - 2 * kHid;
    b3[j] = j < kOut ? th[P.b3 + j] : 0.0f;
  }
}

static int image_elems(const ImgLayout& L) { return kHid * L.ld1 + kHid * kLdh + kOutPad * kLdh + 2 * kHid + kOutPad; }

// Seeded uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) initialisation; parameter
// j of the network's own (compact) order draws counter j, padding stays 0.
__global__ void k_init_params(float* __restrict__ th, ParamLayout P, int n_in, int plain, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.total) return;
  const int j = plain ? paper_index(i, P, n_in) : i;
  if (j < 0) {
    th[i] = 0.0f;
    return;
  }
  const float fan = i < P.w2 ? (float)n_in : (i < P.w3 || !plain ? (float)kHid : (float)kPaperH2);
  const float bound = 1.0f / sqrtf(fan);
  const float u = u24_hi(sm_at(sm_at(sm_at(seed, kStreamInit), 0ull), (uint64_t)j));
  th[i] = -bound + u * (bound + bound);
}

// Copy the image into shared memory (16-byte vectors).
__device__ __forceinline__ void stage_image(uint8_t* dst, const uint8_t* __restrict__ src, int bytes) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = __ldg(s + i);
}

// The same through the bulk-copy engine: thread 0 issues the copies (image
// bytes are a multiple of 16, both ends 16-byte aligned) on the mbarrier
// `bar` (initialised by the caller with one arrival), every thread waits
// for its phase `parity` (bounded).  CTA-wide; false when the copy did not
// complete within the bound.
constexpr int kStageChunk = 32 * 1024;
__device__ __forceinline__ bool stage_image_bulk(uint8_t* dst, const uint8_t* __restrict__ src, int bytes,
                                                 uint64_t* bar, uint32_t parity, uint32_t tries) {
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (uint32_t)bytes);
    for (int off = 0; off < bytes; off += kStageChunk)
      bulk_g2s(dst + off, src + off, (uint32_t)min(kStageChunk, bytes - off), bar);
  }
  return __syncthreads_and(mbar_wait(bar, parity, tries));
}

// Pointers into a shared-memory copy of the image.
struct QW {
  const bf16* W1;
  const bf16* W2;
  const bf16* W3;
  const float* b1;
  const float* b2;
  const float* b3;
  int k1, ld1;
};
__device__ __forceinline__ QW qw_at(const uint8_t* base, const ImgLayout& L) {
  QW w;
  w.W1 = reinterpret_cast<const bf16*>(base + L.w1);
  w.W2 = reinterpret_cast<const bf16*>(base + L.w2);
  w.W3 = reinterpret_cast<const bf16*>(base + L.w3);
  w.b1 = reinterpret_cast<const float*>(base + L.b1);
  w.b2 = reinterpret_cast<const float*>(base + L.b2);
  w.b3 = reinterpret_cast<const float*>(base + L.b3);
  w.k1 = L.k1;
  w.ld1 = L.ld1;
  return w;
}

// One hidden layer for R = 16 * MT rows and R warps: Hout[R][256] =
// bf16(ReLU(Xin * W^T + b)).  The 32 output n-tiles of 8 columns are spread
// over the warps (32 / R per warp), each warp covering all MT m-tiles so
// that one B fragment serves MT MMAs.
template <int MT>
__device__ __forceinline__ void hidden_layer(const bf16* Xin, int ldx, int kdim, const bf16* W, int ldw,
                                             const float* b, bf16* Hout, int warp, int lane) {
  constexpr int kWarps = 16 * MT;
  constexpr int kNt = 32 / kWarps;
  const int g = lane >> 2, q = lane & 3;
#pragma unroll
  for (int t = 0; t < kNt; ++t) {
    const int n0 = 8 * (warp + kWarps * t);
    float acc[MT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) acc[mt][0] = acc[mt][1] = acc[mt][2] = acc[mt][3] = 0.f;
    for (int k0 = 0; k0 < kdim; k0 += 16) {
      uint32_t b0, b1;
      load_b_col(b0, b1, W, ldw, k0, n0, lane);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t a[4];
        load_a_row(a, Xin, ldx, 16 * mt, k0, lane);
        mma_bf16(acc[mt], a, b0, b1);
      }
    }
    const int n = n0 + 2 * q;
    const float bn = b[n], bn1 = b[n + 1];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const int r0 = 16 * mt + g;
      *reinterpret_cast<uint32_t*>(Hout + r0 * kLdh + n) =
          pack_bf16x2(fmaxf(acc[mt][0] + bn, 0.f), fmaxf(acc[mt][1] + bn1, 0.f));
      *reinterpret_cast<uint32_t*>(Hout + (r0 + 8) * kLdh + n) =
          pack_bf16x2(fmaxf(acc[mt][2] + bn, 0.f), fmaxf(acc[mt][3] + bn1, 0.f));
    }
  }
}

// Head for the 16 rows of m-tile mt (one warp): O[16][8] = H2 * W3^T + b3
// (FP32), two accumulator chains (even / odd k-steps) summed in a fixed order.
__device__ __forceinline__ void head_layer(const bf16* H2, const QW& w, float* O, int mt, int lane) {
  const int g = lane >> 2, q = lane & 3;
  float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < kHid; k0 += 32) {
    uint32_t a[4], b0, b1;
    load_a_row(a, H2, kLdh, 16 * mt, k0, lane);
    load_b_col(b0, b1, w.W3, kLdh, k0, 0, lane);
    mma_bf16(acc0, a, b0, b1);
    load_a_row(a, H2, kLdh, 16 * mt, k0 + 16, lane);
    load_b_col(b0, b1, w.W3, kLdh, k0 + 16, 0, lane);
    mma_bf16(acc1, a, b0, b1);
  }
  const int n = 2 * q;
  const int r0 = 16 * mt + g;
  O[r0 * kOutPad + n] = (acc0[0] + acc1[0]) + w.b3[n];
  O[r0 * kOutPad + n + 1] = (acc0[1] + acc1[1]) + w.b3[n + 1];
  O[(r0 + 8) * kOutPad + n] = (acc0[2] + acc1[2]) + w.b3[n];
  O[(r0 + 8) * kOutPad + n + 1] = (acc0[3] + acc1[3]) + w.b3[n + 1];
}

// Full forward of a tile of 16 * MT rows by 16 * MT warps (contains block
// barriers; every thread of the block must call it).
template <int MT = 1>
__device__ __forceinline__ void mlp_tile(const QW& w, const bf16* X, bf16* H1, bf16* H2, float* O, int warp,
                                         int lane) {
  hidden_layer<MT>(X, w.ld1, w.k1, w.W1, w.ld1, w.b1, H1, warp, lane);
  __syncthreads();
  hidden_layer<MT>(H1, kLdh, kHid, w.W2, kLdh, w.b2, H2, warp, lane);
  __syncthreads();
  if (warp < MT) head_layer(H2, w, O, warp, lane);
  __syncthreads();
}

__device__ __forceinline__ void group_barrier(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// The forward of one 16-row tile by a group of 16 warps that synchronise
// among themselves on named barrier `bar` (the other warps of the CTA run
// on); wg = the warp's index in its group.
__device__ __forceinline__ void mlp_tile_group(const QW& w, const bf16* X, bf16* H1, bf16* H2, float* O, int wg,
                                               int lane, int bar) {
  hidden_layer<1>(X, w.ld1, w.k1, w.W1, w.ld1, w.b1, H1, wg, lane);
  group_barrier(bar, 512);
  hidden_layer<1>(H1, kLdh, kHid, w.W2, kLdh, w.b2, H2, wg, lane);
  group_barrier(bar, 512);
  if (wg == 0) head_layer(H2, w, O, 0, lane);
  group_barrier(bar, 512);
}

// Dueling combine and greedy action of one row of head outputs:
// Q_a = (V + A_a) - mean(A), argmax with the lowest index on ties.
__device__ __forceinline__ uint32_t greedy_action(const float* o, float* qv = nullptr, int plain = 0) {
  if (plain) {
    // the paper's network: the outputs are the Q-values
    uint32_t best = 0;
    float bq = o[0];
    if (qv) qv[0] = bq;
#pragma unroll
    for (int a = 1; a < kOut - 1; ++a) {
      if (qv) qv[a] = o[a];
      if (o[a] > bq) {
        bq = o[a];
        best = (uint32_t)a;
      }
    }
    return best;
  }
  const float V = o[0];
  const float meanA = ((((o[1] + o[2]) + o[3]) + o[4]) + o[5]) / 5.0f;
  uint32_t best = 0;
  float bq = (V + o[1]) - meanA;
  if (qv) qv[0] = bq;
#pragma unroll
  for (int a = 1; a < kOut - 1; ++a) {
    const float qa = (V + o[1 + a]) - meanA;
    if (qv) qv[a] = qa;
    if (qa > bq) {
      bq = qa;
      best = (uint32_t)a;
    }
  }
  return best;
}

// This warp's observation row (lane share `o`) into a BF16 tile row.
__device__ __forceinline__ void obs_to_tile(bf16* row, const ObsRegs& o, int B, int lane) {
  if (lane < B) row[lane] = __float2bfloat16_rn(o.b0);
  if (lane + 32 < B) row[lane + 32] = __float2bfloat16_rn(o.b1);
  if (lane < 5) row[B + lane] = __float2bfloat16_rn(o.ex);
}

// ------------------------------------------------ tcgen05 batched forward
// Q[M][5] of obs[M][n_in] on the fifth-generation tensor cores, 128 rows per
// tile.  A persistent CTA (one per SM) holds all weights in shared memory
// (W1, W2, W3: one set of bulk asynchronous copies (TMA) from a copy of the
// online network in the tensor cores' layout, k_tc_image) and the whole
// 512-column tensor memory.  Per tile: the threads convert the 128 input
// rows to BF16 (X, shared memory); one thread issues the MMAs of a layer
// (tcgen05.mma, FP32 accumulators in tensor memory) and commits them to an
// mbarrier; the eight warps read the accumulators back (tcgen05.ld; warps w
// and w + 4 take the rows of lane quarter w % 4 and half of the columns
// each), add the bias, apply ReLU, round to BF16 and store the pairs back
// into the first half of the columns they read (tcgen05.st): the hidden
// activations never leave tensor memory and are the A operand of the next
// layer's MMAs.  Tensor-memory columns:
//   [0, 256)   layer 1 accumulators; H1 in [0, 64) (units 0..127) and [128, 192) (128..255)
//   [256, 512) layer 2 accumulators; H2 in [256, 320) and [384, 448); head accumulators at 320
// The tensor cores run the next tile's layer 1 beside this tile's layer-2
// epilogue, and this tile's head beside the next tile's layer-1 epilogue;
// only layer 2 (N = 256) is waited for by all warps.
// Shared memory: X 128 x k1 | W1 256 x k1 | W2 256 x 256 | W3 16 x 256,
// in the canonical K-major layout of sg_tc.cuh.  Same BF16 recipe as the
// mma.sync kernels (BF16 inputs, weights and hidden activations, FP32 sums);
// only the summation order differs.
constexpr int kTcRows = 128;
constexpr uint32_t kTcTries = 1u << 24;  // bound of every mbarrier wait (polls)
// The launch takes the whole shared memory of an SM (one CTA per SM either
// way), so that every descriptor-addressed byte lies inside the allocation.
constexpr uint32_t kTcSmemLaunch = 227u * 1024u - 4096u;

struct TcSmem {
  uint32_t x, w1, w2, w3, bytes;
};
__host__ __device__ inline uint32_t tc_up(uint32_t v) { return (v + 1023u) & ~1023u; }
__host__ __device__ inline TcSmem tc_smem(int k1) {
  TcSmem t;
  t.x = 0;
  t.w1 = tc_up(t.x + (uint32_t)(kTcRows * k1 * 2));
  t.w2 = tc_up(t.w1 + (uint32_t)(kHid * k1 * 2));
  t.w3 = tc_up(t.w2 + (uint32_t)(kHid * kHid * 2));
  t.bytes = tc_up(t.w3 + (uint32_t)(16 * kHid * 2));
  return t;
}
// k1 <= 80 (n_in <= 69): 197 KB, inside the launch's shared memory
static_assert(kTcRows * 80 * 2 + 1024 + kHid * 80 * 2 + kHid * kHid * 2 + 16 * kHid * 2 + 1024 <= kTcSmemLaunch,
              "tcgen05 forward: operands exceed the shared memory");
// The weight copy in global memory: blocks identical to their shared-memory
// images, so that each is one bulk copy.
// For the fused rollout also W1 in two 128-row halves and W2 in four
// 64-row quarters, and for the batched forward W2 as one 256-row operand
// (each its own canonical operand).
struct TcImg {
  uint32_t w1, w2a, w2b, w3, w1h, w2q, w2f, bytes;
};
__host__ __device__ inline TcImg tc_img(int k1) {
  TcImg t;
  t.w1 = 0;
  t.w2a = (uint32_t)(kHid * k1 * 2);
  t.w2b = t.w2a + 128u * kHid * 2u;
  t.w3 = t.w2b + 128u * kHid * 2u;
  t.w1h = t.w3 + 16u * kHid * 2u;
  t.w2q = t.w1h + (uint32_t)(kHid * k1 * 2);
  t.w2f = t.w2q + (uint32_t)(kHid * kHid * 2);
  t.bytes = t.w2f + (uint32_t)(kHid * kHid * 2);
  return t;
}

// The online weights from the BF16 image (rows of ld1 / kLdh elements) into
// the canonical layout: W1 (256 rows), W2 rows 0..127 and 128..255 (two
// 128-row operands), W3 (16 rows, 6 used).
__global__ void k_tc_image(const uint8_t* __restrict__ img, ImgLayout L, uint8_t* __restrict__ out) {
  const TcImg T = tc_img(L.k1);
  const int n1 = kHid * (L.k1 / 8), n2 = kHid * (kHid / 8), n3 = 16 * (kHid / 8);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n1 + n2 + n3; c += gridDim.x * blockDim.x) {
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    uint32_t dst;
    if (c < n1) {
      const int n = c % kHid, kg = c / kHid;
      v = __ldg(reinterpret_cast<const uint4*>(img + L.w1 + ((size_t)n * L.ld1 + kg * 8) * 2));
      dst = T.w1 + kmajor_offset(n, kg * 8, kHid);
      // the same chunk in its 128-row half
      *reinterpret_cast<uint4*>(out + T.w1h + (uint32_t)((n >> 7) * 128 * L.k1 * 2) +
                                kmajor_offset(n & 127, kg * 8, 128)) = v;
    } else if (c < n1 + n2) {
      const int j = c - n1, n = j % kHid, kg = j / kHid;
      v = __ldg(reinterpret_cast<const uint4*>(img + L.w2 + ((size_t)n * kLdh + kg * 8) * 2));
      dst = n < 128 ? T.w2a + kmajor_offset(n, kg * 8, 128) : T.w2b + kmajor_offset(n - 128, kg * 8, 128);
      // in its 64-row quarter and in the 256-row operand
      *reinterpret_cast<uint4*>(out + T.w2q + (uint32_t)((n >> 6) * 64 * kHid * 2) +
                                kmajor_offset(n & 63, kg * 8, 64)) = v;
      *reinterpret_cast<uint4*>(out + T.w2f + kmajor_offset(n, kg * 8, kHid)) = v;
    } else {
      const int j = c - n1 - n2, n = j % 16, kg = j / 16;
      if (n < kOutPad) v = __ldg(reinterpret_cast<const uint4*>(img + L.w3 + ((size_t)n * kLdh + kg * 8) * 2));
      dst = T.w3 + kmajor_offset(n, kg * 8, 16);
    }
    *reinterpret_cast<uint4*>(out + dst) = v;
  }
}

// Hidden-layer epilogue: this thread's row r = 32 (warp % 4) + lane, columns
// [128 (warp / 4), + 128) of the accumulator plus bias, ReLU, rounded to BF16
// into the H operand.
__device__ __forceinline__ void tc_epilogue_hidden(uint32_t tacc, const float* bias, uint8_t* hs,
                                                   int warp, int lane) {
  const int quarter = warp & 3, r = quarter * 32 + lane, c0 = (warp >> 2) * 128;
  for (int c = c0; c < c0 + 128; c += 32) {
    float v[32];
    tmem_ld32(tacc + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = c + 8 * g + 2 * j;
        w[j] = pack_bf16x2(fmaxf(v[8 * g + 2 * j] + bias[k], 0.f), fmaxf(v[8 * g + 2 * j + 1] + bias[k + 1], 0.f));
      }
      *reinterpret_cast<uint4*>(hs + kmajor_offset(r, c + 8 * g, kTcRows)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// Epilogue warps of the batched forward: four per lane quarter (warp w
// takes lanes 32 (w % 4) .. and the kTfCols accumulator columns of group
// w / 4).
constexpr int kTfEpiWarps = 16;
constexpr int kTfEpiThreads = kTfEpiWarps * 32;
constexpr int kTfThreads = kTfEpiThreads + 32;  // + the MMA-issue warp
constexpr int kTfCols = kHid / (kTfEpiWarps / 4);
static_assert(kTfCols % 32 == 0, "each epilogue warp's columns hold whole 16-column chunks and head accumulators");

// Hidden-layer epilogue in tensor memory: this thread's lane (row
// 32 (warp % 4) + lane), accumulator columns [tacc + kTfCols g, + kTfCols) for
// g = warp / 4, plus the bias, ReLU, rounded to BF16 pairs and stored over the
// first half of those columns (units kTfCols g + 2 c, + 1 in column
// tacc + kTfCols g + c).  The load of the next 16 columns is in flight while
// a chunk is converted; a chunk's 8 output columns lie below every column
// still to be read, and each load completes before the columns it frees are
// written.  Returns once the stores have completed.
__device__ __forceinline__ void tc_epilogue_tmem(uint32_t tacc, const float* bias, int warp) {
  constexpr int kChunks = kTfCols / 16;
  const uint32_t t = tacc + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * kTfCols);
  const float4* b4 = reinterpret_cast<const float4*>(bias + (warp >> 2) * kTfCols);
  uint32_t r[2][16];
  tmem_ld16_nowait(t, r[0]);
  tmem_ld_wait();
#pragma unroll
  for (int ch = 0; ch < kChunks; ++ch) {
    if (ch + 1 < kChunks) tmem_ld16_nowait(t + (uint32_t)(16 * (ch + 1)), r[(ch + 1) & 1]);
    const uint32_t(&v)[16] = r[ch & 1];
    uint32_t w[8];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 bb = b4[4 * ch + j];
      w[2 * j] = pack_bf16x2_relu(__uint_as_float(v[4 * j]) + bb.x, __uint_as_float(v[4 * j + 1]) + bb.y);
      w[2 * j + 1] = pack_bf16x2_relu(__uint_as_float(v[4 * j + 2]) + bb.z, __uint_as_float(v[4 * j + 3]) + bb.w);
    }
    tmem_st8(t + (uint32_t)(8 * ch), w);
    if (ch + 1 < kChunks) tmem_ld_wait();
  }
  tmem_st_wait();
}
// Tensor-memory column (relative to the layer's accumulators) of K step ks
// of the packed activations, and of head accumulator q (four of 16 columns
// in the halves the epilogue leaves free).
__host__ __device__ constexpr uint32_t tf_a_col(int ks) {
  return (uint32_t)((ks / (kTfCols / 16)) * kTfCols + (ks % (kTfCols / 16)) * 8);
}
__host__ __device__ constexpr uint32_t tf_head_col(int q) {
  return (uint32_t)(kTfCols / 2 + (q / (kTfCols / 32)) * kTfCols + (q % (kTfCols / 32)) * 16);
}

// One layer from a tensor-memory A operand (the packed activations of
// tc_epilogue_tmem with accumulators at column a, K = 256):
// D[d] = A x B^T for B in shared memory of Rb rows (K-major, canonical);
// one thread.
__device__ __forceinline__ void tc_layer_ta(uint32_t d, uint32_t a, uint32_t b_smem, int Rb) {
  const uint32_t idesc = idesc_bf16_f32(kTcRows, Rb);
  const uint32_t lb = (uint32_t)Rb * 16;
#pragma unroll 1
  for (int ks = 0; ks < kHid / 16; ++ks)
    tc_mma_bf16_ta(d, a + tf_a_col(ks), smem_desc(b_smem + (uint32_t)ks * 2 * lb, lb, 128), idesc, ks > 0 ? 1u : 0u);
}

// Input rows of a tile into the X operand (BF16, zero padded) in two steps:
// tc_fetch_x loads this thread's values (the kTfEpiThreads / 128 threads of
// a row take interleaved 8-column groups, at most kTcMaxGroups each),
// tc_store_x converts and stores them.
constexpr int kTcXStride = kTfEpiThreads / kTcRows;
constexpr int kTcMaxGroups = (80 / 8 + kTcXStride - 1) / kTcXStride;
struct TcXRegs {
  float v[kTcMaxGroups][8];
};
__device__ __forceinline__ void tc_fetch_x(TcXRegs& x, const float* __restrict__ obs, const ImgLayout& L, int M,
                                           int tile, int tid) {
  const int row = tid & (kTcRows - 1), grow = tile * kTcRows + row, ng = L.k1 / 8;
  const float* src = obs + (long long)grow * L.n_in;
#pragma unroll
  for (int it = 0; it < kTcMaxGroups; ++it) {
    const int kg = (tid >> 7) + kTcXStride * it;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = kg * 8 + j;
      x.v[it][j] = (kg < ng && grow < M && k < L.n_in) ? __ldg(src + k) : 0.0f;
    }
  }
}
__device__ __forceinline__ void tc_store_x(uint8_t* xs, const TcXRegs& x, const ImgLayout& L, int tid) {
  const int row = tid & (kTcRows - 1), ng = L.k1 / 8;
#pragma unroll
  for (int it = 0; it < kTcMaxGroups; ++it) {
    const int kg = (tid >> 7) + kTcXStride * it;
    if (kg < ng)
      *reinterpret_cast<uint4*>(xs + kmajor_offset(row, kg * 8, kTcRows)) =
          make_uint4(pack_bf16x2(x.v[it][0], x.v[it][1]), pack_bf16x2(x.v[it][2], x.v[it][3]),
                     pack_bf16x2(x.v[it][4], x.v[it][5]), pack_bf16x2(x.v[it][6], x.v[it][7]));
  }
  fence_async_smem();
}

// Warps 0..15 run the epilogues, convert the inputs and write Q; warp 16
// (one lane) copies the weights and issues every MMA, so that the issue, which
// waits while the tensor cores' queue is full, never holds up an epilogue.
// The two sides meet on mbarriers, one phase per tile each: bar_x (X
// stored), bar_h1 (H1 stored and the previous tile's head read), bar_h2 (H2
// stored), and the MMA commits bar_l1, bar_l2, bar_hd (layer 1, layer 2,
// head complete).  Order on the tensor cores per tile t: layer 2 (t) once H1
// (t) is stored and the head of t - 1 is read; layer 1 (t + 1) once layer 2
// (t) is complete and X (t + 1) is stored; the head (t) once H2 (t) is stored.
__global__ void __launch_bounds__(kTfThreads, 1) k_qnet_forward_tc(const uint8_t* __restrict__ img,
                                                                const uint8_t* __restrict__ timg, ImgLayout L,
                                                                const float* __restrict__ obs, int M,
                                                                float* __restrict__ qout) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ uint64_t bar_w, bar_l1, bar_l2, bar_hd, bar_x, bar_h1, bar_h2, bar_drain;
  __shared__ uint32_t tslot;
  __shared__ int s_fail;
  __shared__ __align__(16) float sb1[kHid];
  __shared__ __align__(16) float sb2[kHid];
  __shared__ float sb3[kOutPad];
  const TcSmem T = tc_smem(L.k1);
  const TcImg G = tc_img(L.k1);
  uint8_t* xs = tsm + T.x;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ntiles = (M + kTcRows - 1) / kTcRows;
  // this CTA's tiles: blockIdx.x + i gridDim.x, i < my_tiles
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  for (int i = tid; i < kHid; i += kTfThreads) {
    sb1[i] = __ldg(reinterpret_cast<const float*>(img + L.b1) + i);
    sb2[i] = __ldg(reinterpret_cast<const float*>(img + L.b2) + i);
  }
  if (tid < kOutPad) sb3[tid] = __ldg(reinterpret_cast<const float*>(img + L.b3) + tid);
  if (warp == 0) tmem_alloc(&tslot, 512);
  if (tid == 0) {
    mbar_init(&bar_w, 1);
    mbar_init(&bar_l1, 1);
    mbar_init(&bar_l2, 1);
    mbar_init(&bar_hd, 1);
    mbar_init(&bar_drain, 1);
    mbar_init(&bar_x, kTfEpiThreads);
    mbar_init(&bar_h1, kTfEpiThreads);
    mbar_init(&bar_h2, kTfEpiThreads);
    s_fail = 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tslot, tacc2 = tacc + 256u;
  volatile int* fail = &s_fail;
  if (warp == kTfEpiThreads / 32) {
    if ((tid & 31) == 0 && my_tiles > 0) {
      // ---- MMA issue
      const uint32_t sx = smem_u32(xs), sw1 = smem_u32(tsm + T.w1), sw2 = smem_u32(tsm + T.w2),
                     sw3 = smem_u32(tsm + T.w3);
      auto issue_l1 = [&]() {
        const uint32_t idesc = idesc_bf16_f32(kTcRows, kHid);
        const uint32_t la = kTcRows * 16, lb = kHid * 16;
        for (int ks = 0; ks < L.k1 / 16; ++ks)
          tc_mma_bf16(tacc, smem_desc(sx + (uint32_t)ks * 2 * la, la, 128),
                      smem_desc(sw1 + (uint32_t)ks * 2 * lb, lb, 128), idesc, ks > 0 ? 1u : 0u);
        tc_commit(&bar_l1);
      };
      // the resident weights: W1, W2 (one 256-row operand), W3
      mbar_expect_tx(&bar_w, G.w2a + kHid * kHid * 2u + 16u * kHid * 2u);
      bulk_g2s(tsm + T.w1, timg + G.w1, G.w2a, &bar_w);
      bulk_g2s(tsm + T.w2, timg + G.w2f, kHid * kHid * 2u, &bar_w);
      bulk_g2s(tsm + T.w3, timg + G.w3, 16u * kHid * 2u, &bar_w);
      bool ok = mbar_wait_or_fail(&bar_w, 0, kTcTries, fail) && mbar_wait_or_fail(&bar_x, 0, kTcTries, fail);
      if (ok) {
        tc_fence_after();
        issue_l1();
      }
      for (int it = 0; ok && it < my_tiles; ++it) {
        const uint32_t par = (uint32_t)it & 1u;
        // layer 2 (t): D[256, 512) = H1 W2^T, N = 256
        ok = mbar_wait_or_fail(&bar_h1, par, kTcTries, fail);
        if (!ok) break;
        tc_fence_after();
        tc_layer_ta(tacc2, tacc, sw2, kHid);
        tc_commit(&bar_l2);
        // layer 1 (t + 1) over H1 (t), once layer 2 (t) has read it
        if (it + 1 < my_tiles) {
          ok = mbar_wait_or_fail(&bar_x, par ^ 1u, kTcTries, fail) && mbar_wait_or_fail(&bar_l2, par, kTcTries, fail);
          if (!ok) break;
          tc_fence_after();
          issue_l1();
        }
        // head (t): N = 16 (6 used) into four accumulators in layer-2
        // columns the epilogue has read and left free, K step ks into
        // accumulator ks % 4
        ok = mbar_wait_or_fail(&bar_h2, par, kTcTries, fail);
        if (!ok) break;
        tc_fence_after();
        {
          const uint32_t idesc = idesc_bf16_f32(kTcRows, 16);
#pragma unroll 1
          for (int ks = 0; ks < kHid / 16; ++ks)
            tc_mma_bf16_ta(tacc2 + tf_head_col(ks & 3), tacc2 + tf_a_col(ks),
                           smem_desc(sw3 + (uint32_t)ks * 2 * 256, 256, 128), idesc, ks >= 4 ? 1u : 0u);
        }
        tc_commit(&bar_hd);
      }
      // every MMA of this thread, and the weight copies, complete before the
      // tensor memory is freed (bounded waits)
      tc_commit(&bar_drain);
      mbar_wait(&bar_drain, 0, kTcTries);
      mbar_wait(&bar_w, 0, kTcTries);
    }
  } else {
    // ---- epilogues, inputs, read-out (warps 0..7)
    bool ok = true;
    const int row = tid & (kTcRows - 1);
    auto wait = [&](uint64_t* bar, uint32_t par) {
      ok = __all_sync(0xffffffffu, ok && mbar_wait_or_fail(bar, par, kTcTries, fail));
      if (ok) tc_fence_after();
    };
    // Q rows of local tile i from the four head accumulators (NaN where a
    // wait ran out)
    auto write_rows = [&](int i) {
      uint32_t h[4][8];
      if (ok && warp < 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) tmem_ld8_nowait(tacc2 + tf_head_col(q) + ((uint32_t)(warp * 32) << 16), h[q]);
        tmem_ld_wait();
      }
      const int grow = ((int)blockIdx.x + i * (int)gridDim.x) * kTcRows + row;
      if (warp < 4 && grow < M) {
        float qv[5];
        if (ok) {
          float o[kOut];
#pragma unroll
          for (int j = 0; j < kOut; ++j)
            o[j] = ((__uint_as_float(h[0][j]) + __uint_as_float(h[1][j])) +
                    (__uint_as_float(h[2][j]) + __uint_as_float(h[3][j]))) +
                   sb3[j];
          greedy_action(o, qv, L.plain);
        } else {
#pragma unroll
          for (int a = 0; a < 5; ++a) qv[a] = __int_as_float(0x7fc00000);
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) qout[(long long)grow * 5 + a] = qv[a];
      }
    };
    TcXRegs xr;
    if (my_tiles > 0) {
      tc_fetch_x(xr, obs, L, M, blockIdx.x, tid);
      tc_store_x(xs, xr, L, tid);
      mbar_arrive(&bar_x);
    }
    for (int it = 0; it < my_tiles; ++it) {
      const uint32_t par = (uint32_t)it & 1u;
      wait(&bar_l1, par);
      if (ok) tc_epilogue_tmem(tacc, sb1, warp);  // H1 over the layer-1 accumulators
      if (it > 0) {
        wait(&bar_hd, par ^ 1u);
        write_rows(it - 1);
        // the read-out (warps 0..3) is on the critical path: the other
        // warps' input loads start after it
        asm volatile("bar.sync 1, %0;\n" ::"n"(kTfEpiThreads) : "memory");
      }
      tc_fence_before();
      mbar_arrive(&bar_h1);
      // X is free (layer 1 of t is complete): the next tile's inputs while layer 2 runs
      if (ok && it + 1 < my_tiles) {
        tc_fetch_x(xr, obs, L, M, (int)blockIdx.x + (it + 1) * (int)gridDim.x, tid);
        tc_store_x(xs, xr, L, tid);
        mbar_arrive(&bar_x);
      }
      wait(&bar_l2, par);
      if (ok) tc_epilogue_tmem(tacc2, sb2, warp);  // H2 over the layer-2 accumulators
      tc_fence_before();
      mbar_arrive(&bar_h2);
    }
    if (my_tiles > 0) {
      wait(&bar_hd, (uint32_t)(my_tiles - 1) & 1u);
      write_rows(my_tiles - 1);
    }
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tacc, 512);
}

// VEM eps-greedy rollout with the network fused in: per step, the 16 envs of
// a group write their observations to a BF16 tile, the tile goes through the
// network on the tensor cores, every env takes argmax Q or (with probability
// eps_i) the random action, then steps; the transition is appended to the
// replay ring.  One warp per env; 16 envs per group, MT groups per CTA
// sharing the weight image.  The groups synchronise only among themselves
// (named barriers), so one group's env step overlaps the other's network.
template <int MT, bool kDyn>
__global__ void __launch_bounds__(512 * MT, 1)
    k_rollout_q(const __grid_constant__ DevCfg c, SimPtrs p, const uint8_t* __restrict__ img, ImgLayout L, int K,
                const float* __restrict__ eps, ReplayDev rp, int use_replay, const int* __restrict__ order, int epc,
                float* __restrict__ obs_out,
                float* __restrict__ obs_seq, uint8_t* __restrict__ act_seq, float* __restrict__ rew_seq,
                uint8_t* __restrict__ done_seq) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sw = smem;
  bf16* X = reinterpret_cast<bf16*>(smem + L.bytes);
  constexpr int kRows = 16 * MT;
  bf16* H1 = X + kRows * L.ld1;
  bf16* H2 = H1 + kRows * kLdh;
  float* O = reinterpret_cast<float*>(H2 + kRows * kLdh);
  stage_image(sw, img, L.bytes);
  for (int i = threadIdx.x; i < kRows * L.ld1; i += blockDim.x) X[i] = __float2bfloat16_rn(0.0f);
  const QW w = qw_at(sw, L);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp >> 4, wg = warp & 15, bar = 1 + grp;
  bf16* Xg = X + grp * 16 * L.ld1;
  bf16* H1g = H1 + grp * 16 * kLdh;
  bf16* H2g = H2 + grp * 16 * kLdh;
  float* Og = O + grp * 16 * kOutPad;
  // CTAs take envs grouped by map, so that one CTA's scans share cache lines;
  // epc <= kRows envs per CTA (fewer than the tile when that spreads the
  // envs over more SMs; the tile's other rows stay zero)
  const int slot = blockIdx.x * epc + warp;
  const bool live = warp < epc && slot < c.n_envs;
  const int env = live ? order[slot] : 0;
  const long long n = c.n_envs;
  EnvConst k;
  Env s;
  ObsRegs o;
  o.b0 = o.b1 = o.ex = 0.0f;
  float eps_i = 0.0f;
  uint64_t akey = 0;
  // dynamic obstacles: lane o holds disc o, every lane the centres
  Obst b = {0.0f, 0.0f, 0.0f, 0.0f};
  Discs dsc;
  if (live) {
    k = env_const(c, p, env, lane);
    s = load_env(p, env);
    if (kDyn) {
      if (lane < c.n_dyn) b = load_obst(p, lane, env);
      gather_discs(c, b, dsc);
    }
    const Noise z = noise_for(k, s.sigma, s.ep_id, s.ep_step, lane);
    Aux aux;
    observe<kDyn>(c, k, s, z, lane, o, aux, &dsc);  // the current observation, from the state
    eps_i = eps[env];
    akey = sm_at(sm_at(c.seed, kStreamAction), (uint64_t)env);
  }
  const unsigned long long rbase = use_replay ? *rp.steps : 0ull;
  uint32_t ra_batch = 0, ex_batch = 0;
  __syncthreads();
  for (int i = 0; i < K; ++i) {
    if (live) obs_to_tile(Xg + wg * L.ld1, o, c.B, lane);
    group_barrier(bar, 512);
    mlp_tile_group(w, Xg, H1g, H2g, Og, wg, lane, bar);
    if (!live) continue;
    if ((i & 31) == 0) {
      // lane l draws the random action and the exploration uniform of step t + l
      const uint64_t h = sm_at(akey, (uint64_t)(s.t + (uint32_t)lane));
      ra_batch = (uint32_t)(sm_at(h, 0ull) >> 32) % (uint32_t)c.n_actions;
      ex_batch = __ballot_sync(kFull, u24_hi(sm_at(h, 1ull)) < eps_i);
    }
    const uint32_t ra = __shfl_sync(kFull, ra_batch, i & 31);
    const bool explore = (ex_batch >> (i & 31)) & 1u;
    const uint32_t greedy = greedy_action(Og + wg * kOutPad, nullptr, L.plain);
    const uint32_t a = explore ? ra : greedy;
    long long e = 0;
    float* srow = nullptr;
    float* s2row = nullptr;
    if (use_replay) {
      e = (long long)((rbase + (unsigned long long)i) % (unsigned long long)rp.slots) * rp.n_envs + env;
      srow = rp.s + e * rp.obs_dim;
      s2row = rp.s2 + e * rp.obs_dim;
      write_obs(srow, o, c.B, lane);
    }
    const StepOut r = env_step<kDyn>(c, p, k, s, a, lane, o, s2row, &b, &dsc);
    if (use_replay) {
      if (!r.done) write_obs(s2row, o, c.B, lane);
      if (lane == 0) {
        rp.a[e] = (uint8_t)a;
        rp.r[e] = r.rew;
        rp.term[e] = (r.done & 3u) ? 1 : 0;
      }
    }
    if (obs_seq) write_obs(obs_seq + ((long long)i * n + env) * c.obs_dim, o, c.B, lane);
    if (lane == 0) {
      if (act_seq) act_seq[i * n + env] = (uint8_t)a;
      if (rew_seq) rew_seq[i * n + env] = r.rew;
      if (done_seq) done_seq[i * n + env] = (uint8_t)r.done;
    }
  }
  if (live) {
    if (obs_out) write_obs(obs_out + (long long)env * c.obs_dim, o, c.B, lane);
    if (lane == 0) store_env(p, env, s);
    if (kDyn && lane < c.n_dyn) store_obst(p, lane, env, b);
  }
}

// ---------------------------------------- tcgen05 fused eps-greedy rollout
// For large env counts: 128 envs per CTA form one 128-row tile of the
// network.  Per step the network runs on the tile on the tensor cores
// (tcgen05 MMAs into 256 tensor-memory columns, epilogues split over the 8
// warps of each lane quarter), warps 0-3 take the greedy actions from the
// head, the first 16 warps step the tile's envs the way sg_sim_step does (8
// envs per warp, one per lane: the scalar part, lane_step), and then every
// warp takes whole-warp scans row by row from a shared counter, writing the
// next observation as the tile's BF16 row and the FP32 outputs and ring
// entries.  Same VEM draws, same simulator values as k_rollout_q; the Q
// values differ from it only in the summation order.
//
// Shared memory is kept small (136 KB) so that L1 keeps room for the maps the
// scans read: the input tile (at most 20 KB) and the step records (16 KB,
// from byte 32 K) live inside the hidden-activation buffer, which holds H1
// and H2 during the network only, and all of W1 (two 128-row halves) and W2
// (four 32 KB pieces: the K halves of its two 128-row halves) stream through
// two 32 KB buffers by bulk copies
// every step, each copy issued as soon as its buffer's previous MMAs are
// done (both W1 halves during the env steps, the first two W2 pieces during
// the layer-1 epilogue); W3 stays.
constexpr int kQtEnvs = 128;
constexpr int kQtWarps = 32;
constexpr int kQtThreads = kQtWarps * 32;
constexpr uint32_t kQtBuf = 32u * 1024u;
constexpr uint32_t kQtRecOff = 32u * 1024u;
// The env steps of a tile (the scalar part, lane_step) run on the first
// kQtEnvs / kQtStepLanes warps, kQtStepLanes envs per warp (one per lane):
// 16 warps of 8 envs measured fastest (32 x 4: 406.2, 16 x 8: 414.5,
// 8 x 16: 411.4, 4 x 32: 400.5 M env-steps/s at 65,536 envs).
constexpr int kQtStepLanes = 8;  // records in the activation buffer (input tile: 256 k1 <= 20 KB)
static_assert(kQtRecOff + kQtEnvs * 128u <= (uint32_t)(kQtEnvs * kHid * 2), "records fit the activation buffer");

struct QtSmem {
  uint32_t hx, b0, b1, w3, bytes;
};
__host__ __device__ inline QtSmem qt_smem() {
  QtSmem t;
  t.hx = 0;
  t.b0 = (uint32_t)(kQtEnvs * kHid * 2);
  t.b1 = t.b0 + kQtBuf;
  t.w3 = t.b1 + kQtBuf;
  t.bytes = t.w3 + 16u * kHid * 2u;
  return t;
}

// Epilogue of a hidden layer by 32 warps: warp w takes the rows of lane
// quarter w % 4 and columns [32 (w / 4), + 32).
__device__ __forceinline__ void qt_epilogue(uint32_t tacc, const float* bias, uint8_t* hs, int warp, int lane) {
  const int quarter = warp & 3, r = quarter * 32 + lane, c = (warp >> 2) * 32;
  float v[32];
  tmem_ld32(tacc + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = c + 8 * g + 2 * j;
      w[j] = pack_bf16x2(fmaxf(v[8 * g + 2 * j] + bias[k], 0.f), fmaxf(v[8 * g + 2 * j + 1] + bias[k + 1], 0.f));
    }
    *reinterpret_cast<uint4*>(hs + kmajor_offset(r, c + 8 * g, kQtEnvs)) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// This lane's share of an observation row into row r of the BF16 input tile.
__device__ __forceinline__ void qt_obs_to_tile(uint8_t* xs, int r, float b0, float b1, float ex, int B, int lane) {
  if (lane < B) *reinterpret_cast<bf16*>(xs + kmajor_offset(r, lane, kQtEnvs)) = __float2bfloat16_rn(b0);
  if (lane + 32 < B) *reinterpret_cast<bf16*>(xs + kmajor_offset(r, lane + 32, kQtEnvs)) = __float2bfloat16_rn(b1);
  if (lane < 5) *reinterpret_cast<bf16*>(xs + kmajor_offset(r, B + lane, kQtEnvs)) = __float2bfloat16_rn(ex);
}

// The weight stream of the fused rollout, run by the CTA's thread 0: chunk
// copies into two buffers (one mbarrier each for the copy, one for the MMAs
// that read the buffer) with every copy and every MMA group waited exactly
// once, in order.
struct QtStream {
  uint64_t* ld;    // [2] copy complete
  uint64_t* mm;    // [2] MMAs reading the buffer complete
  uint8_t* buf[2];
  uint32_t pl[2], pm[2];
  bool ld_out[2], mm_out[2];
  bool ok;
  // copy `bytes` from src into buffer b once its previous MMAs are done
  __device__ __forceinline__ void load(int b, const void* src, uint32_t bytes) {
    if (!ok) return;
    if (mm_out[b]) {
      ok = mbar_wait(&mm[b], pm[b], kTcTries);
      pm[b] ^= 1u;
      mm_out[b] = false;
      if (!ok) return;
    }
    mbar_expect_tx(&ld[b], bytes);
    bulk_g2s(buf[b], src, bytes, &ld[b]);
    ld_out[b] = true;
  }
  // MMAs D[tacc] (+)= A x buffer b^T (Rb rows, K; A from its K step ks0,
  // onto D when acc), then commits: the buffer's barrier, and the layer
  // barrier when `last`
  __device__ __forceinline__ void mma(int b, uint32_t tacc, const uint8_t* a, int Rb, int K, uint64_t* layer,
                                      bool last, int ks0 = 0, bool acc = false) {
    if (!ok) return;
    if (ld_out[b]) {
      ok = mbar_wait(&ld[b], pl[b], kTcTries);
      pl[b] ^= 1u;
      ld_out[b] = false;
      if (!ok) return;
    }
    tc_fence_after();
    const uint32_t idesc = idesc_bf16_f32(kQtEnvs, Rb);
    const uint32_t sa = smem_u32(a), sb = smem_u32(buf[b]);
    const uint32_t la = kQtEnvs * 16, lb = (uint32_t)Rb * 16;
    for (int ks = 0; ks < K / 16; ++ks)
      tc_mma_bf16(tacc, smem_desc(sa + (uint32_t)(ks0 + ks) * 2 * la, la, 128),
                  smem_desc(sb + (uint32_t)ks * 2 * lb, lb, 128), idesc, (acc || ks > 0) ? 1u : 0u);
    tc_commit(&mm[b]);
    mm_out[b] = true;
    if (last) tc_commit(layer);
  }
  // bounded waits for whatever is still in flight
  __device__ __forceinline__ void drain() {
    for (int b = 0; b < 2; ++b) {
      if (mm_out[b]) mbar_wait(&mm[b], pm[b], kTcTries);
      if (ld_out[b]) mbar_wait(&ld[b], pl[b], kTcTries);
    }
  }
};

// State of env i through L2: with time slicing another SM may have written
// it during this launch.
__device__ __forceinline__ Env load_env_l2(const SimPtrs& p, int i) {
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

__device__ __forceinline__ unsigned qt_ld_acquire(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void qt_st_release(unsigned* a, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;\n" ::"l"(a), "r"(v) : "memory");
}
constexpr unsigned kQtWaitIters = 1u << 22;  // x ~256 ns sleeps: about a second

// Time slicing (sync != null): a resident grid takes (segment of seg steps,
// 128-env block) items in segment-major order from a device counter; an item
// waits (bounded) until the previous segment of its block is published, and
// takes its first observation from the replay ring (the entry the previous
// segment wrote), or scans it when there is no ring.  sync: [nblk] segments
// done per block, item counter, abort word; zero at launch.
__global__ void __launch_bounds__(kQtThreads, 1)
    k_rollout_q_tc(const __grid_constant__ DevCfg c, SimPtrs p, const uint8_t* __restrict__ img,
                   const uint8_t* __restrict__ timg, ImgLayout L, int K, const float* __restrict__ eps, ReplayDev rp,
                   int use_replay, const int* __restrict__ order, int seg, unsigned* __restrict__ sync,
                   float* __restrict__ obs_out, float* __restrict__ obs_seq, uint8_t* __restrict__ act_seq,
                   float* __restrict__ rew_seq, uint8_t* __restrict__ done_seq) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ uint64_t bar_ld[2], bar_mm[2], bar_layer;
  __shared__ uint32_t tslot;
  __shared__ int item_sh;
  __shared__ int ok_sh;
  __shared__ int greedy[kQtEnvs];
  __shared__ uint8_t act_sh[kQtEnvs];
  __shared__ int scan_next;
  __shared__ Env env_sh[kQtEnvs];                 // the tile's env states within a segment
  __shared__ unsigned long long akey_sh[kQtEnvs];  // their action-stream keys
  __shared__ float sb1[kHid], sb2[kHid], sb3[kOutPad];
  const QtSmem T = qt_smem();
  const TcImg G = tc_img(L.k1);
  uint8_t* hx = tsm + T.hx;  // the input tile, then H1, then H2
  uint8_t* w3s = tsm + T.w3;
  StepScanRec* rec = reinterpret_cast<StepScanRec*>(tsm + T.hx + kQtRecOff);  // during the env steps only
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long n = c.n_envs;
  const int nblk = (int)((n + kQtEnvs - 1) / kQtEnvs);
  const int seglen = seg > 0 ? seg : K;
  const int nseg = (K + seglen - 1) / seglen;
  const long long nitems = (long long)nblk * nseg;
  const uint32_t w1h_bytes = 128u * (uint32_t)L.k1 * 2u, w2q_bytes = 64u * kHid * 2u;
  for (int i = tid; i < kHid; i += kQtThreads) {
    sb1[i] = __ldg(reinterpret_cast<const float*>(img + L.b1) + i);
    sb2[i] = __ldg(reinterpret_cast<const float*>(img + L.b2) + i);
  }
  if (tid < kOutPad) sb3[tid] = __ldg(reinterpret_cast<const float*>(img + L.b3) + tid);
  for (int i = tid; i < (int)(16u * kHid * 2u / 16u); i += kQtThreads)
    reinterpret_cast<uint4*>(w3s)[i] = __ldg(reinterpret_cast<const uint4*>(timg + G.w3) + i);
  if (warp == 0) tmem_alloc(&tslot, 256);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_ld[b], 1);
      mbar_init(&bar_mm[b], 1);
    }
    mbar_init(&bar_layer, 1);
    ok_sh = 1;
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tacc = tslot;
  QtStream S;  // meaningful in thread 0
  S.ld = bar_ld;
  S.mm = bar_mm;
  S.buf[0] = tsm + T.b0;
  S.buf[1] = tsm + T.b1;
  S.pl[0] = S.pl[1] = S.pm[0] = S.pm[1] = 0u;
  S.ld_out[0] = S.ld_out[1] = S.mm_out[0] = S.mm_out[1] = false;
  S.ok = true;
  uint32_t player = 0;  // phase of the layer barrier
  bool layer_out = false, ok = true;
  const unsigned long long rbase = use_replay ? *rp.steps : 0ull;
  const int B = c.B;
  const int row0 = warp * 4;
  for (int iter = 0;; ++iter) {
    // ---- the next item: a segment of one 128-env block ----
    if (tid == 0) {
      long long it;
      if (!sync)
        it = iter == 0 ? (long long)blockIdx.x : nitems;
      else
        it = (!ok || __ldcg(&sync[nblk + 1])) ? nitems : (long long)atomicAdd(&sync[nblk], 1u);
      if (sync && it < nitems && it >= nblk) {
        const unsigned need = (unsigned)(it / nblk);
        unsigned w = 0;
        while (qt_ld_acquire(&sync[it % nblk]) < need) {
          if (++w > kQtWaitIters || qt_ld_acquire(&sync[nblk + 1])) {
            atomicOr(p.status, SG_DEV_TIMEOUT);
            atomicExch(&sync[nblk + 1], 1u);
            it = nitems;
            break;
          }
          __nanosleep(256);
        }
      }
      item_sh = (ok && it < nitems) ? (int)it : -1;
    }
    __syncthreads();
    const int item = item_sh;
    __syncthreads();  // item_sh is rewritten by the next iteration
    if (item < 0) break;
    const int blk = item % nblk, s0 = (item / nblk) * seglen, s1 = min(K, s0 + seglen);
    // the segment's first observation: four rows per warp (row0 .. row0 + 3)
    const int slot0 = blk * kQtEnvs + row0;
    const int nv = max(0, min(4, (int)n - slot0));
    const bool live = lane < nv;
    const int env = live ? order[slot0 + lane] : 0;
    // the env-step lanes: row srow of the tile
    const bool stepper = warp < kQtEnvs / kQtStepLanes;
    const int srow = warp * kQtStepLanes + lane;
    const bool slive = stepper && lane < kQtStepLanes && (long long)blk * kQtEnvs + srow < n;
    const int senv = slive ? order[blk * kQtEnvs + srow] : 0;
    // the tile: zero (padding columns, rows without an env), then the first
    // observation of the segment
    for (int i = tid; i < kQtEnvs * L.k1 / 8; i += kQtThreads)
      reinterpret_cast<uint4*>(hx)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    if (s0 > 0 && use_replay) {
      const long long sl = (long long)((rbase + (unsigned long long)s0) % (unsigned long long)rp.slots);
      for (int e = 0; e < nv; ++e) {
        const int ie = __shfl_sync(kFull, env, e);
        const float* src = rp.s + (sl * rp.n_envs + ie) * rp.obs_dim;
        for (int k = lane; k < c.obs_dim; k += 32)
          *reinterpret_cast<bf16*>(hx + kmajor_offset(row0 + e, k, kQtEnvs)) = __float2bfloat16_rn(__ldcg(src + k));
      }
    } else {
      if (live) lane_observe(c, p, env, load_env_l2(p, env), rec[row0 + lane]);
      __syncwarp();
      for (int e = 0; e < nv; ++e) {
        const StepScanRec& r = rec[row0 + e];
        float b0, b1;
        scan_env(c, p, p.maps[r.map], r.nb, r.stepb, r.ax, r.ay, r.aphi, r.asigma,
                 ((uint64_t)r.anhi << 32) | r.anlo, lane, b0, b1);
        qt_obs_to_tile(hx, row0 + e, b0, b1, lane < 5 ? r.exa[lane] : 0.0f, B, lane);
        if (use_replay) {
          const long long sl = (long long)((rbase + (unsigned long long)s0) % (unsigned long long)rp.slots);
          write_row(rp.s + (sl * rp.n_envs + r.env) * rp.obs_dim, b0, b1, r.exa, B, lane);
        }
      }
    }
    fence_async_smem();
    for (int t = s0; t < s1; ++t) {
      // ---- the network on the tile of observations t ----
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // layer 1: two 128-unit halves of W1 through the buffers (normally
      // loaded during the previous env steps), then the two K-half pieces of
      // W2's first 128 rows into them as soon as each half's MMAs are done
      if (tid == 0) {
        if (!S.ld_out[0]) S.load(0, timg + G.w1h, w1h_bytes);
        if (!S.ld_out[1]) S.load(1, timg + G.w1h + w1h_bytes, w1h_bytes);
        S.mma(0, tacc, hx, 128, L.k1, &bar_layer, false);
        S.mma(1, tacc + 128u, hx, 128, L.k1, &bar_layer, true);
        S.load(0, timg + G.w2a, w2q_bytes);
        S.load(1, timg + G.w2a + w2q_bytes, w2q_bytes);
        if (!S.ok) ok_sh = 0;
      }
      layer_out = true;
      __syncthreads();  // ok_sh as thread 0 left it
      ok = __syncthreads_and(ok_sh && mbar_wait(&bar_layer, player, kTcTries));
      if (!ok) break;
      player ^= 1u;
      layer_out = false;
      tc_fence_after();
      qt_epilogue(tacc, sb1, hx, warp, lane);  // H1 over the input tile
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // layer 2: two 128-unit halves (N = 128: an MMA of M = 128 costs about
      // as much at N = 64 as at 128), each from the two 32 KB K-half pieces
      // of its rows through the buffers (piece c: K steps 8 c .. 8 c + 7);
      // the second half's pieces are both in flight before either is needed
      if (tid == 0) {
        S.mma(0, tacc, hx, 128, kHid / 2, &bar_layer, false, 0, false);
        S.mma(1, tacc, hx, 128, kHid / 2, &bar_layer, false, 8, true);
        S.load(0, timg + G.w2b, w2q_bytes);
        S.load(1, timg + G.w2b + w2q_bytes, w2q_bytes);
        S.mma(0, tacc + 128u, hx, 128, kHid / 2, &bar_layer, false, 0, false);
        S.mma(1, tacc + 128u, hx, 128, kHid / 2, &bar_layer, true, 8, true);
        if (!S.ok) ok_sh = 0;
      }
      layer_out = true;
      __syncthreads();  // ok_sh as thread 0 left it
      ok = __syncthreads_and(ok_sh && mbar_wait(&bar_layer, player, kTcTries));
      if (!ok) break;
      player ^= 1u;
      layer_out = false;
      tc_fence_after();
      qt_epilogue(tacc, sb2, hx, warp, lane);  // H2 over H1 (layer 2 is complete)
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // head (W3 resident), and the next step's W1 halves into the buffers
      if (tid == 0) {
        tc_fence_after();
        const uint32_t idesc = idesc_bf16_f32(kQtEnvs, 16);
        const uint32_t sa = smem_u32(hx), sw = smem_u32(w3s);
        for (int ks = 0; ks < kHid / 16; ++ks)
          tc_mma_bf16(tacc, smem_desc(sa + (uint32_t)ks * 2 * (kQtEnvs * 16), kQtEnvs * 16, 128),
                      smem_desc(sw + (uint32_t)ks * 2 * 256, 256, 128), idesc, ks > 0 ? 1u : 0u);
        tc_commit(&bar_layer);
        if (t + 1 < s1) {
          S.load(0, timg + G.w1h, w1h_bytes);
          S.load(1, timg + G.w1h + w1h_bytes, w1h_bytes);
        }
        if (!S.ok) ok_sh = 0;
      }
      layer_out = true;
      __syncthreads();  // ok_sh as thread 0 left it
      ok = __syncthreads_and(ok_sh && mbar_wait(&bar_layer, player, kTcTries));
      if (!ok) break;
      player ^= 1u;
      layer_out = false;
      if (warp < 4) {
        float v[32];
        tc_fence_after();
        tmem_ld32(tacc + ((uint32_t)(warp * 32) << 16), v);
        float o[kOut];
#pragma unroll
        for (int j = 0; j < kOut; ++j) o[j] = v[j] + sb3[j];
        greedy[warp * 32 + lane] = (int)greedy_action(o, nullptr, L.plain);
      }
      // the next input tile starts from zero (H2 is dead after the head)
      for (int i = tid; i < kQtEnvs * L.k1 / 8; i += kQtThreads)
        reinterpret_cast<uint4*>(hx)[i] = make_uint4(0u, 0u, 0u, 0u);
      if (tid == 0) scan_next = 0;
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
      // ---- the env steps of the tile: one env per lane of the stepping warps ----
      if (stepper) {
        Env s;
        uint32_t a = 0;
        if (slive) {
          // the state stays in shared memory between the steps of a segment
          // (stored to global memory at its last step)
          s = t == s0 ? load_env_l2(p, senv) : env_sh[srow];
          if (t == s0) akey_sh[srow] = sm_at(sm_at(c.seed, kStreamAction), (uint64_t)senv);
          // VEM (Sec. 3.1.1): with probability eps_i the random action of step t
          const uint64_t h = sm_at(akey_sh[srow], (uint64_t)s.t);
          const uint32_t ra = (uint32_t)(sm_at(h, 0ull) >> 32) % (uint32_t)c.n_actions;
          const bool explore = u24_hi(sm_at(h, 1ull)) < __ldg(eps + senv);
          a = explore ? ra : (uint32_t)greedy[srow];
        }
        const uint32_t d = lane_step(c, p, senv, slive, s, a, rec[slive ? srow : 0], lane);
        if (slive) {
          env_sh[srow] = s;
          if (t + 1 == s1) store_env(p, senv, s);
          act_sh[srow] = (uint8_t)a;
          if (act_seq) act_seq[(long long)t * n + senv] = (uint8_t)a;
          if (done_seq) done_seq[(long long)t * n + senv] = (uint8_t)d;
        }
      }
      // every record of the tile is written; the scans (one or two per env,
      // 16 to 64 beams) are handed out row by row through a shared counter,
      // so that no warp waits at the next step's barrier for a slow one
      __syncthreads();
      const long long slot_t =
          use_replay ? (long long)((rbase + (unsigned long long)t) % (unsigned long long)rp.slots) : 0;
      const long long slot_n =
          use_replay ? (long long)((rbase + (unsigned long long)t + 1ull) % (unsigned long long)rp.slots) : 0;
      const int rows = (int)min((long long)kQtEnvs, n - (long long)blk * kQtEnvs);
      for (;;) {
        int e = 0;
        if (lane == 0) e = atomicAdd(&scan_next, 1);
        e = __shfl_sync(kFull, e, 0);
        if (e >= rows) break;
        const StepScanRec& r = rec[e];
        const int ie = r.env;
        const uint32_t de = r.done;
        const MapDesc m = p.maps[r.map];
        float b0, b1;
        const float mn = scan_env(c, p, m, r.nb, r.stepb, r.ax, r.ay, r.aphi, r.asigma,
                                  ((uint64_t)r.anhi << 32) | r.anlo, lane, b0, b1);
        const float rw = (de & 1u) ? -10.0f : (de & 2u) ? 75.0f : reward_finish(c, r.rpart, mn);
        const uint32_t ae = act_sh[e];
        if (use_replay) {
          // transition t: s2 is the observation after the step, before a reset
          const long long en = slot_t * rp.n_envs + ie;
          write_row(rp.s2 + en * rp.obs_dim, b0, b1, r.exa, B, lane);
          if (lane == 0) {
            rp.a[en] = (uint8_t)ae;
            rp.r[en] = rw;
            rp.term[en] = (de & 3u) ? 1 : 0;
          }
        }
        if (lane == 0 && rew_seq) rew_seq[(long long)t * n + ie] = rw;
        const float* ex = r.exa;
        if (de) {
          scan_env(c, p, m, r.nb, r.stepb, r.bx, r.by, r.bphi, r.bsigma, ((uint64_t)r.bnhi << 32) | r.bnlo, lane,
                   b0, b1);
          ex = r.exb;
        }
        // the observation t + 1: the next tile row, the outputs, the next ring entry's s
        qt_obs_to_tile(hx, e, b0, b1, lane < 5 ? ex[lane] : 0.0f, B, lane);
        if (obs_seq) write_row(obs_seq + ((long long)t * n + ie) * c.obs_dim, b0, b1, ex, B, lane);
        if (t == K - 1 && obs_out) write_row(obs_out + (long long)ie * c.obs_dim, b0, b1, ex, B, lane);
        if (use_replay && t + 1 < K)
          write_row(rp.s + (slot_n * rp.n_envs + ie) * rp.obs_dim, b0, b1, ex, B, lane);
      }
      fence_async_smem();
    }
    if (!ok) {
      if (tid == 0) atomicOr(p.status, SG_DEV_TIMEOUT);
      break;  // CTA-uniform: the launch's outputs from here on are incomplete
    }
    if (!sync) break;
    // publish the block's segment: its env state and ring entries are stored
    __threadfence();
    __syncthreads();
    if (tid == 0) qt_st_release(&sync[blk], (unsigned)(s0 / seglen + 1));
  }
  // free the tensor memory once nothing is in flight (bounded waits)
  if (tid == 0) S.drain();
  if (layer_out && ok_sh) mbar_wait(&bar_layer, player, kTcTries);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_free(tacc, 256);
}

__global__ void k_replay_advance(unsigned long long* steps, int K) { *steps += (unsigned long long)K; }

// ------------------------------------------------------------ learner
// Why a TD step produced no update (bits of a device word cleared at the
// start of every step): a weight-image copy did not complete within its
// bounded wait, or a sample's action index is outside the action table.
// k_adam then writes NaN loss and gradient and leaves the parameters, the
// Adam moments and the image untouched; the step count does not advance.
constexpr unsigned kTdFailCopy = 1u;
constexpr unsigned kTdFailAction = 2u;
// Ring entry of sample i of optimiser step `tstep`: uniform over the
// V = min(steps, slots - reserve) most recently completed slots, so that a
// rollout running concurrently (which writes the next slots) is never read.
// With j = h mod (V n_envs): slot = (steps - 1 - j / n_envs) mod slots,
// env = j mod n_envs.
__device__ __forceinline__ long long sample_entry(unsigned long long seed, unsigned long long tstep, int i,
                                                  const ReplayDev& rp) {
  const unsigned long long st = *rp.steps;
  const unsigned long long usable = (unsigned long long)(rp.slots - rp.reserve);
  const unsigned long long V = st < usable ? st : usable;
  if (V == 0) return -1;
  const uint64_t h = sm_at(sm_at(sm_at(sm_at(seed, kStreamSample), tstep), (uint64_t)i), 0ull);
  const unsigned long long j = h % (V * (unsigned long long)rp.n_envs);
  const unsigned long long back = j / (unsigned long long)rp.n_envs;
  const unsigned long long slot = (st - 1ull - back) % (unsigned long long)rp.slots;
  const long long e = (long long)(slot * (unsigned long long)rp.n_envs + j % (unsigned long long)rp.n_envs);
  return SG_IN_BOUNDS(e >= 0 && e < (long long)rp.slots * rp.n_envs) ? e : -1;
}

// Gather 16 rows of a ring array into a BF16 tile (zero padded).
__device__ __forceinline__ void gather_tile(bf16* X, int ld1, const float* __restrict__ src, const int* rows,
                                            int obs_dim, int warp, int lane) {
  const int e = rows[warp];
  for (int k = lane; k < ld1; k += 32) {
    const float v = (e >= 0 && k < obs_dim) ? src[(long long)e * obs_dim + k] : 0.0f;
    X[warp * ld1 + k] = __float2bfloat16_rn(v);
  }
}

// Double-DQN targets of 16 samples per CTA: a* = argmax_a Q_online(s', a),
// y = r + gamma (1 - term) Q_target(s', a*).  Also records the sampled entries.
__global__ void __launch_bounds__(kThreads, 1)
    k_td_target(const uint8_t* __restrict__ img, const uint8_t* __restrict__ img_t, ImgLayout L, ReplayDev rp,
                unsigned long long seed, const unsigned long long* __restrict__ step, int batch, float gamma,
                float* __restrict__ y, int* __restrict__ idx, unsigned* __restrict__ fail) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sw = smem;
  bf16* X = reinterpret_cast<bf16*>(smem + L.bytes);
  bf16* H1 = X + kTile * L.ld1;
  bf16* H2 = H1 + kTile * kLdh;
  float* O = reinterpret_cast<float*>(H2 + kTile * kLdh);
  __shared__ int rows[kTile];
  __shared__ int astar[kTile];
  __shared__ uint64_t bar_img;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kTile + warp;
  if (lane == 0) {
    rows[warp] = i < batch ? (int)sample_entry(seed, *step, i, rp) : -1;
    if (i < batch) idx[i] = rows[warp];
  }
  if (threadIdx.x == 0) mbar_init(&bar_img, 1);
  __syncthreads();
  // online image (phase 0) while the tile is gathered; a copy that does not
  // complete makes the targets NaN
  bool ok = stage_image_bulk(sw, img, L.bytes, &bar_img, 0u, kTcTries);
  uint32_t phase = 0u;  // the copy in flight
  gather_tile(X, L.ld1, rp.s2, rows, rp.obs_dim, warp, lane);
  __syncthreads();
  if (ok) mlp_tile(qw_at(sw, L), X, H1, H2, O, warp, lane);
  if (lane == 0) astar[warp] = (int)greedy_action(O + warp * kOutPad, nullptr, L.plain);
  fence_async_smem();  // this thread's reads of the online image before the bulk copy overwrites it
  __syncthreads();
  // the target image over it (phase 1)
  if (ok) {
    phase = 1u;
    ok = stage_image_bulk(sw, img_t, L.bytes, &bar_img, 1u, kTcTries);
  }
  if (ok) mlp_tile(qw_at(sw, L), X, H1, H2, O, warp, lane);
  if (!ok) {
    if (threadIdx.x == 0) {
      atomicOr(fail, kTdFailCopy);
      // the copy that timed out may still be writing shared memory: give it
      // one more bounded wait before the CTA exits
      mbar_wait(&bar_img, phase, kTcTries);
    }
    if (lane == 0 && i < batch) y[i] = __int_as_float(0x7fc00000);
  }
  if (lane == 0 && i < batch && ok) {
    float qv[5];
    greedy_action(O + warp * kOutPad, qv, L.plain);
    const int e = rows[warp];
    const float r = e >= 0 ? rp.r[e] : 0.0f;
    const float nt = (e >= 0 && rp.term[e]) ? 0.0f : 1.0f;
    y[i] = r + gamma * nt * qv[astar[warp]];
  }
}

// Loss and gradient of 16 samples per CTA.  Forward of Q_online(s) keeping
// the activations, delta = Q(s, a) - y, dL/dQ(s,a) = clip(delta, -1, 1) / B,
// back through the dueling combine, W3, ReLU, W2, ReLU, W1.  The CTA's
// parameter gradient (and Huber sum) goes to its own row of `partial`, so
// that the reduction order is fixed.
__global__ void __launch_bounds__(kThreads, 1)
    k_td_grad(const uint8_t* __restrict__ img, ImgLayout L, ParamLayout P, ReplayDev rp,
              const int* __restrict__ idx, const float* __restrict__ y, int batch, float* __restrict__ partial,
              unsigned* __restrict__ fail) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sw = smem;
  bf16* S = reinterpret_cast<bf16*>(smem + L.bytes);
  bf16* H1 = S + kTile * L.ld1;
  bf16* H2 = H1 + kTile * kLdh;  // becomes dZ2 after the head gradient
  bf16* D1 = H2 + kTile * kLdh;  // dZ1
  float* O = reinterpret_cast<float*>(D1 + kTile * kLdh);
  float* DO = O + kTile * kOutPad;  // dL/d(head outputs) [16][8]
  __shared__ int rows[kTile];
  __shared__ float hub[kTile];
  __shared__ uint64_t bar_img;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  const int i = blockIdx.x * kTile + warp;
  if (lane == 0) rows[warp] = i < batch ? idx[i] : -1;
  if (threadIdx.x == 0) mbar_init(&bar_img, 1);
  __syncthreads();
  if (!stage_image_bulk(sw, img, L.bytes, &bar_img, 0u, kTcTries)) {
    // the image copy did not complete: no update this step (k_adam reads the
    // flag); one more bounded wait for the copy before the CTA exits
    if (threadIdx.x == 0) {
      atomicOr(fail, kTdFailCopy);
      mbar_wait(&bar_img, 0u, kTcTries);
    }
    return;
  }
  gather_tile(S, L.ld1, rp.s, rows, rp.obs_dim, warp, lane);
  __syncthreads();
  const QW w = qw_at(sw, L);
  mlp_tile(w, S, H1, H2, O, warp, lane);
  // dL/dQ and back through Q_a = V + A_a - mean(A)
  if (lane == 0) {
    float qv[5];
    greedy_action(O + warp * kOutPad, qv, L.plain);
    const int e = rows[warp];
    float gq = 0.0f, hl = 0.0f;
    if (e >= 0) {
      int a = rp.a[e];
      float d;
      if (a >= 5) {
        // outside the action table: no loss term, and no update this step
        atomicOr(fail, kTdFailAction);
        a = 0;
        d = __int_as_float(0x7fc00000);
      } else {
        d = qv[a] - y[i];
      }
      const float ad = fabsf(d);
      hl = ad <= 1.0f ? 0.5f * d * d : ad - 0.5f;
      // a NaN target (a failed target copy) stays NaN through the clip
      gq = (isnan(d) ? d : fminf(fmaxf(d, -1.0f), 1.0f)) / (float)batch;
      if (L.plain) {
        for (int k = 0; k < 5; ++k) DO[warp * kOutPad + k] = k == a ? gq : 0.0f;
        DO[warp * kOutPad + 5] = 0.0f;
      } else {
        DO[warp * kOutPad + 0] = gq;
        for (int k = 0; k < 5; ++k) DO[warp * kOutPad + 1 + k] = (k == a ? gq : 0.0f) - gq / 5.0f;
      }
    } else {
      for (int k = 0; k < 6; ++k) DO[warp * kOutPad + k] = 0.0f;
    }
    DO[warp * kOutPad + 6] = 0.0f;
    DO[warp * kOutPad + 7] = 0.0f;
    hub[warp] = hl;
  }
  __syncthreads();
  float* pg = partial + (long long)blockIdx.x * partial_stride(P.total);
  // head gradient on the CUDA cores: dW3[o][j] = sum_s DO[s][o] H2[s][j],
  // db3[o] = sum_s DO[s][o]; dH2 = DO W3 (BF16 W3 as in the forward), masked
  // by the ReLU into dZ2 (written over H2 after a barrier)
  const int tid = threadIdx.x;
  float dz2v[kTile];
  if (tid < kHid) {
    const int j = tid;
    float acc[kOut];
    for (int o = 0; o < kOut; ++o) acc[o] = 0.0f;
    for (int s = 0; s < kTile; ++s) {
      const float h = __bfloat162float(H2[s * kLdh + j]);
      for (int o = 0; o < kOut; ++o) acc[o] += DO[s * kOutPad + o] * h;
    }
    for (int o = 0; o < kOut; ++o) pg[P.w3 + o * kHid + j] = acc[o];
    float db2 = 0.0f;
    for (int s = 0; s < kTile; ++s) {
      float dh = 0.0f;
      for (int o = 0; o < kOut; ++o) dh += DO[s * kOutPad + o] * __bfloat162float(w.W3[o * kLdh + j]);
      const float v = __bfloat162float(H2[s * kLdh + j]) > 0.0f ? dh : 0.0f;
      dz2v[s] = v;
      db2 += v;
    }
    pg[P.b2 + j] = db2;
  }
  if (tid < kOut) {
    float acc = 0.0f;
    for (int s = 0; s < kTile; ++s) acc += DO[s * kOutPad + tid];
    pg[P.b3 + tid] = acc;
  }
  if (tid == 0) {
    float acc = 0.0f;
    for (int s = 0; s < kTile; ++s) acc += hub[s];
    pg[P.total] = acc;
  }
  __syncthreads();
  if (tid < kHid)
    for (int s = 0; s < kTile; ++s) H2[s * kLdh + tid] = __float2bfloat16_rn(dz2v[s]);
  __syncthreads();
  bf16* DZ2 = H2;
  // dW2[m][n] = sum_s dZ2[s][m] H1[s][n]: M = N = 256, K = 16 -> 512 tiles,
  // 32 per warp (A = dZ2^T, B = H1, both stored sample-major)
  for (int t = warp; t < 16 * 32; t += kTile) {
    const int m0 = (t >> 5) * 16, n0 = (t & 31) * 8;
    uint32_t a[4], b0, b1;
    load_a_col(a, DZ2, kLdh, m0, 0, lane);
    load_b_row(b0, b1, H1, kLdh, 0, n0, lane);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_bf16(acc, a, b0, b1);
    float* dst = pg + P.w2;
    *reinterpret_cast<float2*>(dst + (m0 + g) * kHid + n0 + 2 * q) = make_float2(acc[0], acc[1]);
    *reinterpret_cast<float2*>(dst + (m0 + g + 8) * kHid + n0 + 2 * q) = make_float2(acc[2], acc[3]);
  }
  // dH1 = dZ2 W2 (B = W2 stored [out][in] -> "row" layout), masked -> dZ1
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int n0 = 8 * warp + 128 * half;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < kHid; k0 += 16) {
      uint32_t a[4], b0, b1;
      load_a_row(a, DZ2, kLdh, 0, k0, lane);
      load_b_row(b0, b1, w.W2, kLdh, k0, n0, lane);
      mma_bf16(acc, a, b0, b1);
    }
    const int n = n0 + 2 * q;
    const bool m00 = __bfloat162float(H1[g * kLdh + n]) > 0.f, m01 = __bfloat162float(H1[g * kLdh + n + 1]) > 0.f;
    const bool m10 = __bfloat162float(H1[(g + 8) * kLdh + n]) > 0.f;
    const bool m11 = __bfloat162float(H1[(g + 8) * kLdh + n + 1]) > 0.f;
    *reinterpret_cast<uint32_t*>(D1 + g * kLdh + n) = pack_bf16x2(m00 ? acc[0] : 0.f, m01 ? acc[1] : 0.f);
    *reinterpret_cast<uint32_t*>(D1 + (g + 8) * kLdh + n) = pack_bf16x2(m10 ? acc[2] : 0.f, m11 ? acc[3] : 0.f);
    // db1 needs the FP32 values: reduce the 16 rows of this fragment column
    float c0 = (m00 ? acc[0] : 0.f) + (m10 ? acc[2] : 0.f);
    float c1 = (m01 ? acc[1] : 0.f) + (m11 ? acc[3] : 0.f);
    for (int off = 4; off < 32; off <<= 1) {
      c0 += __shfl_xor_sync(kFull, c0, off);
      c1 += __shfl_xor_sync(kFull, c1, off);
    }
    if (g == 0) {
      pg[P.b1 + n] = c0;
      pg[P.b1 + n + 1] = c1;
    }
  }
  __syncthreads();
  // dW1[m][k] = sum_s dZ1[s][m] S[s][k]: M = 256, N = k1, K = 16
  const int nt1 = L.k1 / 8;
  for (int t = warp; t < 16 * nt1; t += kTile) {
    const int m0 = (t / nt1) * 16, n0 = (t % nt1) * 8;
    uint32_t a[4], b0, b1;
    load_a_col(a, D1, kLdh, m0, 0, lane);
    load_b_row(b0, b1, S, L.ld1, 0, n0, lane);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    mma_bf16(acc, a, b0, b1);
    float* dst = pg + P.w1;
    const int c0 = n0 + 2 * q, c1 = c0 + 1;
    if (c0 < L.n_in) {
      dst[(m0 + g) * L.n_in + c0] = acc[0];
      dst[(m0 + g + 8) * L.n_in + c0] = acc[2];
    }
    if (c1 < L.n_in) {
      dst[(m0 + g) * L.n_in + c1] = acc[1];
      dst[(m0 + g + 8) * L.n_in + c1] = acc[3];
    }
  }
}

// Sum the per-CTA partials in CTA order, Adam (Kingma & Ba) on the FP32
// master, and the BF16 image entry of each parameter.  The step counter is
// read here and advanced by k_step_advance afterwards.
__global__ void k_adam(float* __restrict__ th, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ partial, int nblk, ParamLayout P, ImgLayout L, uint8_t* __restrict__ img,
                       const unsigned long long* __restrict__ step, float lr, float b1, float b2, float eps,
                       float* __restrict__ loss, float* __restrict__ grad_out, int batch,
                       const unsigned* __restrict__ fail) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (*fail) {
    // no usable gradient this step: NaN out, parameters and moments unchanged
    const float qnan = __int_as_float(0x7fc00000);
    if (i == 0 && loss) *loss = qnan;
    if (grad_out && i < P.total) {
      const int j = L.plain ? paper_index(i, P, L.n_in) : i;
      if (j >= 0) grad_out[j] = qnan;
    }
    return;
  }
  if (i == 0 && loss) {
    float acc = 0.0f;
    for (int b = 0; b < nblk; ++b) acc += partial[(long long)b * partial_stride(P.total) + P.total];
    *loss = acc / (float)batch;
  }
  if (i >= P.total) return;
  float gsum = 0.0f;
  for (int b = 0; b < nblk; ++b) gsum += partial[(long long)b * partial_stride(P.total) + i];
  if (grad_out) {
    const int j = L.plain ? paper_index(i, P, L.n_in) : i;
    if (j >= 0) grad_out[j] = gsum;
  }
  if (lr == 0.0f) return;
  const float t = (float)(*step + 1ull);
  const float mi = b1 * m[i] + (1.0f - b1) * gsum;
  const float vi = b2 * v[i] + (1.0f - b2) * gsum * gsum;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.0f - powf(b1, t));
  const float vh = vi / (1.0f - powf(b2, t));
  const float nth = th[i] - lr * mh / (sqrtf(vh) + eps);
  th[i] = nth;
  // image entry
  const bf16 hv = __float2bfloat16_rn(nth);
  if (i < P.b1) {
    const int r = i / L.n_in, k = i % L.n_in;
    reinterpret_cast<bf16*>(img + L.w1)[r * L.ld1 + k] = hv;
  } else if (i < P.w2) {
    reinterpret_cast<float*>(img + L.b1)[i - P.b1] = nth;
  } else if (i < P.b2) {
    const int j = i - P.w2;
    reinterpret_cast<bf16*>(img + L.w2)[(j / kHid) * kLdh + j % kHid] = hv;
  } else if (i < P.w3) {
    reinterpret_cast<float*>(img + L.b2)[i - P.b2] = nth;
  } else if (i < P.b3) {
    const int j = i - P.w3;
    reinterpret_cast<bf16*>(img + L.w3)[(j / kHid) * kLdh + j % kHid] = hv;
  } else {
    reinterpret_cast<float*>(img + L.b3)[i - P.b3] = nth;
  }
}

__global__ void k_step_advance(unsigned long long* step, const unsigned* __restrict__ fail) {
  if (!*fail) *step += 1ull;
}

// Target network <- online network when the optimiser step count is a
// multiple of `every` (checked on the device, so the call can be replayed
// from a CUDA graph).
__global__ void k_target_sync(const unsigned long long* __restrict__ step, int every, const float* __restrict__ th,
                              float* __restrict__ tgt, const uint8_t* __restrict__ img, uint8_t* __restrict__ img_t,
                              int P, int img_words, const uint8_t* __restrict__ tc, uint8_t* __restrict__ tc_t,
                              int tc_words) {
  if (every <= 0 || (*step % (unsigned long long)every) != 0ull) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) tgt[i] = th[i];
  if (i < img_words) reinterpret_cast<uint32_t*>(img_t)[i] = reinterpret_cast<const uint32_t*>(img)[i];
  if (i < tc_words) reinterpret_cast<uint32_t*>(tc_t)[i] = reinterpret_cast<const uint32_t*>(tc)[i];
}


// ------------------------------------------------ tcgen05 learner (batch >= 128)
// The TD step for large batches on the fifth-generation tensor cores, in
// 128-sample tiles (one per CTA, 8 warps, the whole shared memory, 512
// tensor-memory columns):
//   k_td_target_tc: per (network, tile) job the forward of Q_online(s') or
//     Q_target(s') (the fused rollout's layer order, weights streamed through
//     two 32 KB buffers); the Q-values go to global memory.
//   k_td_grad_tc: per tile y = r + gamma (1 - term) Q_target(s', argmax
//     Q_online(s')), the forward on s keeping H1 and H2, dQ -> dO (dueling
//     combine), dW3 / db3 / dH2 / dZ2 / db2 on the CUDA cores, then on the
//     tensor cores dW2 = dZ2^T H1, dH1 = dZ2 W2^T (-> dZ1, db1) and
//     dW1 = dZ1^T X; the tile's gradient goes to its own partial row, so the
//     reduction (k_adam, in tile order) is fixed.
// The weight-gradient and backpropagation products read their operands
// transposed: a K-major tile [rows][cols] (core matrices of 8 rows x 16
// bytes, LBO = rows x 16 between 8-column groups, SBO = 128 between 8-row
// groups) is, for the transposed product, an MN-major operand whose core
// matrices are the same 128 bytes (8 consecutive MN elements per 16-byte
// row, 8 K rows): SBO = rows x 16 between 8-element MN groups, LBO = 128
// between 8-row K groups, and the instruction descriptor's transpose bit of
// that operand set.  The same BF16 recipe as the mma.sync learner (BF16
// weights, activations and backpropagated dZ, FP32 sums; dW3, db and the
// head on the CUDA cores in FP32).
constexpr int kLtRows = 128;
constexpr int kLtThreads = 256;
// Below this batch the 16-sample mma.sync learner is faster (its CTAs spread
// over more SMs); measured on one GB300: 58 vs 98 us per step at batch 256,
// 120 vs 98 us at 4,096 with the two-kernel tcgen05 learner.
constexpr int kLtMinBatch = 2048;
constexpr uint32_t kLtBuf = 32u * 1024u;

struct LtSmem {
  uint32_t x, h1, h2, b0, b1, dout, bias, bytes;
};
__host__ __device__ inline LtSmem lt_smem(int k1) {
  LtSmem t;
  t.x = 0;
  t.h1 = tc_up((uint32_t)(kLtRows * k1 * 2));
  t.h2 = t.h1 + (uint32_t)(kLtRows * kHid * 2);
  t.b0 = t.h2 + (uint32_t)(kLtRows * kHid * 2);
  t.b1 = t.b0 + kLtBuf;
  t.dout = t.b1 + kLtBuf;                          // dO [128][8] float
  t.bias = t.dout + (uint32_t)(kLtRows * kOutPad * 4);  // b1, b2 [256] float, b3 [8], reduction scratch [4][256]
  t.bytes = t.bias + (uint32_t)((2 * kHid + kOutPad + 4 * kHid) * 4);
  return t;
}

// Instruction descriptor with the operands' major-ness: trans_a / trans_b = 1
// reads A / B MN-major (bits 15 / 16).
__host__ __device__ constexpr uint32_t idesc_bf16_f32_t(int M, int N, int trans_a, int trans_b) {
  return idesc_bf16_f32(M, N) | ((uint32_t)trans_a << 15) | ((uint32_t)trans_b << 16);
}

// nks MMAs of K = 16: A at a0 + ks * ka, B at b0 + ks * kb (shared-memory
// byte addresses), each with its own leading / stride byte offsets.
__device__ __forceinline__ void lt_mma(uint32_t tacc, uint32_t a0, uint32_t lba, uint32_t sba, uint32_t ka,
                                       uint32_t b0, uint32_t lbb, uint32_t sbb, uint32_t kb, uint32_t idesc, int nks,
                                       bool accumulate) {
  for (int ks = 0; ks < nks; ++ks)
    tc_mma_bf16(tacc, smem_desc(a0 + (uint32_t)ks * ka, lba, sba), smem_desc(b0 + (uint32_t)ks * kb, lbb, sbb), idesc,
                (accumulate || ks > 0) ? 1u : 0u);
}

// The two weight buffers of a CTA, run by thread 0: a copy into buffer b
// waits (bounded) until the MMAs that read it are done.
struct LtStream {
  uint64_t* ld;
  uint64_t* mm;
  uint8_t* buf[2];
  uint32_t pl[2], pm[2];
  bool ld_out[2], mm_out[2];
  bool ok;
  __device__ __forceinline__ void load(int b, const void* src, uint32_t bytes) {
    if (!ok) return;
    if (mm_out[b]) {
      ok = mbar_wait(&mm[b], pm[b], kTcTries);
      pm[b] ^= 1u;
      mm_out[b] = false;
      if (!ok) return;
    }
    mbar_expect_tx(&ld[b], bytes);
    bulk_g2s(buf[b], src, bytes, &ld[b]);
    ld_out[b] = true;
  }
  __device__ __forceinline__ bool ready(int b) {
    if (!ok) return false;
    if (ld_out[b]) {
      ok = mbar_wait(&ld[b], pl[b], kTcTries);
      pl[b] ^= 1u;
      ld_out[b] = false;
    }
    if (ok) tc_fence_after();
    return ok;
  }
  __device__ __forceinline__ void done(int b) {
    tc_commit(&mm[b]);
    mm_out[b] = true;
  }
  __device__ __forceinline__ void drain() {
    for (int b = 0; b < 2; ++b) {
      if (mm_out[b]) mbar_wait(&mm[b], pm[b], kTcTries);
      if (ld_out[b]) mbar_wait(&ld[b], pl[b], kTcTries);
    }
  }
};

// Rows of a tile: sample i's ring entry (or -1 past the batch) into X (BF16,
// K-major, zero padded); the two threads of a row take alternate 8-column
// groups.
__device__ __forceinline__ void lt_load_x(uint8_t* xs, const float* __restrict__ src, const int* rows_sh, int n_in,
                                          int k1, int tid) {
  const int row = tid & (kLtRows - 1);
  const int e = rows_sh[row];
  for (int kg = tid >> 7; kg < k1 / 8; kg += 2) {
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = kg * 8 + j;
      v[j] = (e >= 0 && k < n_in) ? __ldg(src + (long long)e * n_in + k) : 0.0f;
    }
    *reinterpret_cast<uint4*>(xs + kmajor_offset(row, kg * 8, kLtRows)) =
        make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
  }
  fence_async_smem();
}

// A CTA-wide barrier that also orders the tensor-core work around it.
__device__ __forceinline__ void lt_sync() {
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

// Thread 0: the two W1 halves of timg into the two buffers (issued before the
// tile's inputs are gathered, so that the copies overlap the gathers).
__device__ __forceinline__ void lt_prefetch_w1(LtStream& S, const uint8_t* __restrict__ timg, const ImgLayout& L) {
  const TcImg G = tc_img(L.k1);
  const uint32_t w1h = 128u * (uint32_t)L.k1 * 2u;
  S.load(0, timg + G.w1h, w1h);
  S.load(1, timg + G.w1h + w1h, w1h);
}

// The forward of one tile (X in xs) through the network whose tensor-core
// image is timg (W1 already on its way, lt_prefetch_w1), the hidden
// activations left in h1s / h2s (BF16, K-major), the head's 16 columns in
// tensor-memory columns [0, 16).  Thread 0 issues the MMAs and copies; every
// thread runs the epilogues.  Returns false when a wait ran out (then
// nothing after it was issued).
__device__ __forceinline__ bool lt_forward(LtStream& S, uint64_t* bar_layer, uint32_t& player, uint32_t tacc,
                                           const uint8_t* __restrict__ timg, const ImgLayout& L, uint8_t* xs,
                                           uint8_t* h1s, uint8_t* h2s, const float* b1, const float* b2, int tid,
                                           bool& layer_out) {
  const TcImg G = tc_img(L.k1);
  const int warp = tid >> 5, lane = tid & 31;
  const uint32_t w2q = 64u * kHid * 2u;
  const uint32_t sx = smem_u32(xs), sh1 = smem_u32(h1s), sh2 = smem_u32(h2s);
  const uint32_t kA = kLtRows * 16u;  // K-group stride of a 128-row K-major tile
  if (tid == 0) {
    // layer 1 in two 128-unit halves (W1 halves in the two buffers)
    for (int h = 0; h < 2; ++h)
      if (S.ready(h)) {
        lt_mma(tacc + 128u * h, sx, kA, 128, 2 * kA, smem_u32(S.buf[h]), 128u * 16u, 128, 2u * 128u * 16u,
               idesc_bf16_f32(kLtRows, 128), L.k1 / 16, false);
        S.done(h);
      }
    if (S.ok) tc_commit(bar_layer);
    // W2 in 32 KB pieces: the two K halves of its first 128 rows follow as
    // soon as the buffers are free
    S.load(0, timg + G.w2a, w2q);
    S.load(1, timg + G.w2a + w2q, w2q);
  }
  layer_out = true;
  bool ok = __syncthreads_and(mbar_wait(bar_layer, player, kTcTries));
  player ^= 1u;
  layer_out = !ok;
  if (!ok) return false;
  tc_fence_after();
  tc_epilogue_hidden(tacc, b1, h1s, warp, lane);
  fence_async_smem();
  lt_sync();
  if (tid == 0) {
    // layer 2 in two 128-unit halves (N = 128: an MMA of M = 128 costs
    // about as much at N = 64 as at 128), each from two 32 KB K-half pieces
    // of its rows (piece c: K steps 8 c .. 8 c + 7, in buffer c); the second
    // half's pieces are copied in as the first half's are consumed
    for (int h = 0; h < 2; ++h)
      for (int c = 0; c < 2; ++c) {
        if (h == 1) S.load(c, timg + G.w2b + (uint32_t)c * w2q, w2q);
        if (S.ready(c)) {
          lt_mma(tacc + 128u * h, sh1 + (uint32_t)(16 * c) * kA, kA, 128, 2 * kA, smem_u32(S.buf[c]), 128u * 16u,
                 128, 2u * 128u * 16u, idesc_bf16_f32(kLtRows, 128), kHid / 32, c > 0);
          S.done(c);
        }
      }
    if (S.ok) tc_commit(bar_layer);
    S.load(0, timg + G.w3, 16u * kHid * 2u);  // the head's weights next
  }
  layer_out = true;
  ok = __syncthreads_and(mbar_wait(bar_layer, player, kTcTries));
  player ^= 1u;
  layer_out = !ok;
  if (!ok) return false;
  tc_fence_after();
  tc_epilogue_hidden(tacc, b2, h2s, warp, lane);
  fence_async_smem();
  lt_sync();
  if (tid == 0) {
    if (S.ready(0)) {
      lt_mma(tacc, sh2, kA, 128, 2 * kA, smem_u32(S.buf[0]), 16u * 16u, 128, 2u * 16u * 16u,
             idesc_bf16_f32(kLtRows, 16), kHid / 16, false);
      S.done(0);
      tc_commit(bar_layer);
    }
  }
  layer_out = true;
  ok = __syncthreads_and(mbar_wait(bar_layer, player, kTcTries));
  player ^= 1u;
  layer_out = !ok;
  if (ok) tc_fence_after();
  return ok;
}

// Sum of this lane's 32 values over the warp's 32 lanes, column by column:
// afterwards lane l holds the sum of column l (fixed butterfly order).
__device__ __forceinline__ float lt_colsum32(float (&v)[32], int lane) {
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const bool upper = (lane & w) != 0;
#pragma unroll
    for (int i = 0; i < w; ++i) {
      const float send = upper ? v[i] : v[i + w];
      const float keep = upper ? v[i + w] : v[i];
      v[i] = keep + __shfl_xor_sync(kFull, send, w);
    }
  }
  return v[0];
}

// Bias vectors of a network's image into shared memory.
__device__ __forceinline__ void lt_biases(const uint8_t* __restrict__ im, const ImgLayout& L, float* b1, float* b2,
                                          float* b3, int tid) {
  for (int i = tid; i < kHid; i += kLtThreads) {
    b1[i] = __ldg(reinterpret_cast<const float*>(im + L.b1) + i);
    b2[i] = __ldg(reinterpret_cast<const float*>(im + L.b2) + i);
  }
  if (tid < kOutPad) b3[tid] = __ldg(reinterpret_cast<const float*>(im + L.b3) + tid);
  __syncthreads();
}

// The tensor-core work of one TD step in one kernel.  CTAs take jobs in start
// order from a device counter: jobs [0, 2 ntiles) are the next-state
// forwards (Q_online(s') of tile t, then Q_target(s') of tile t; Q-values to
// q2[net][i][5], then the tile's counter in sync is raised), jobs
// [2 ntiles, 4 ntiles) the tiles' loss and gradient in two halves per tile
// (role 0: dW3, db3, db2, the loss, dW2; role 1: dH1, db1, dW1), each from its
// own forward on s, into partial[tile].  A gradient job runs its forward
// first and only then waits (bounded) for its tile's two next-state jobs:
// those were taken earlier by CTAs that are running and never wait, so the
// wait ends for any grid size.
// sync: [0] the job counter, [1 + t] next-state jobs done for tile t; zero at
// launch.
__global__ void __launch_bounds__(kLtThreads, 1)
    k_td_tc(const uint8_t* __restrict__ img, const uint8_t* __restrict__ img_t, const uint8_t* __restrict__ timg,
            const uint8_t* __restrict__ timg_t, ImgLayout L, ParamLayout P, ReplayDev rp, unsigned long long seed,
            const unsigned long long* __restrict__ step, int batch, float gamma, float* __restrict__ q2,
            int* __restrict__ idx, unsigned* __restrict__ sync, float* __restrict__ partial,
            unsigned* __restrict__ fail) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ uint64_t bar_ld[2], bar_mm[2], bar_layer;
  __shared__ uint32_t tslot;
  __shared__ int rows_sh[kLtRows];
  __shared__ float y_sh[kLtRows];
  __shared__ float hub_sh[kLtRows / 32];
  __shared__ int job_sh, flag_sh;
  const LtSmem T = lt_smem(L.k1);
  const TcImg G = tc_img(L.k1);
  uint8_t* xs = tsm + T.x;
  uint8_t* h1s = tsm + T.h1;
  uint8_t* h2s = tsm + T.h2;
  float* dout = reinterpret_cast<float*>(tsm + T.dout);
  float* b1 = reinterpret_cast<float*>(tsm + T.bias);
  float* b2 = b1 + kHid;
  float* b3 = b2 + kHid;
  float* red = b3 + kOutPad;  // [4][256] column sums of the four lane quarters
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (batch + kLtRows - 1) / kLtRows;
  const uint32_t w2q = 64u * kHid * 2u;
  const uint32_t kA = kLtRows * 16u;
  const bf16* W3g = reinterpret_cast<const bf16*>(img + L.w3);
  if (warp == 0) tmem_alloc(&tslot, 512);
  if (tid == 0) {
    mbar_init(&bar_ld[0], 1);
    mbar_init(&bar_ld[1], 1);
    mbar_init(&bar_mm[0], 1);
    mbar_init(&bar_mm[1], 1);
    mbar_init(&bar_layer, 1);
  }
  lt_sync();
  const uint32_t tacc = tslot;
  LtStream S;
  S.ld = bar_ld;
  S.mm = bar_mm;
  S.buf[0] = tsm + T.b0;
  S.buf[1] = tsm + T.b1;
  S.pl[0] = S.pl[1] = S.pm[0] = S.pm[1] = 0u;
  S.ld_out[0] = S.ld_out[1] = S.mm_out[0] = S.mm_out[1] = false;
  S.ok = true;
  uint32_t player = 0;
  bool layer_out = false, ok = true;
  const unsigned long long tstep = *step;
  for (;;) {
    if (tid == 0) job_sh = (int)atomicAdd(sync, 1u);
    __syncthreads();
    const int job = job_sh;
    __syncthreads();  // every thread has the job before the next one is taken
    if (job >= 4 * ntiles || !ok) break;
    if (job < 2 * ntiles) {
      const int net = job >= ntiles ? 1 : 0, tile = job - net * ntiles;
      lt_biases(net ? img_t : img, L, b1, b2, b3, tid);
      if (tid == 0) lt_prefetch_w1(S, net ? timg_t : timg, L);
      if (tid < kLtRows) {
        const int i = tile * kLtRows + tid;
        const int e = i < batch ? (int)sample_entry(seed, tstep, i, rp) : -1;
        rows_sh[tid] = e;
        if (net == 0 && i < batch) idx[i] = e;
      }
      __syncthreads();
      lt_load_x(xs, rp.s2, rows_sh, L.n_in, L.k1, tid);
      lt_sync();
      ok = lt_forward(S, &bar_layer, player, tacc, net ? timg_t : timg, L, xs, h1s, h2s, b1, b2, tid, layer_out);
      if (warp < 4) {
        const int i = tile * kLtRows + warp * 32 + lane;
        float v[32];
        if (ok) tmem_ld32(tacc + ((uint32_t)(warp * 32) << 16), v);
        if (i < batch) {
          float qv[5];
          if (ok) {
            float o[kOut];
#pragma unroll
            for (int j = 0; j < kOut; ++j) o[j] = v[j] + b3[j];
            greedy_action(o, qv, L.plain);
          } else {
#pragma unroll
            for (int a = 0; a < 5; ++a) qv[a] = __int_as_float(0x7fc00000);
          }
#pragma unroll
          for (int a = 0; a < 5; ++a) q2[((long long)net * batch + i) * 5 + a] = qv[a];
        }
      }
      // publish (also after a failure, whose Q-values are NaN): the values
      // before the tile's counter (release)
      __threadfence();
      __syncthreads();
      if (tid == 0) atomicAdd(sync + 1 + tile, 1u);
      lt_sync();
      continue;
    }
    // gradient jobs: role 0 of a tile computes dW3, db3, db2, the loss and
    // dW2; role 1 (on another CTA, from the same forward) dH1, db1 and dW1
    const int role = job >= 3 * ntiles ? 1 : 0;
    const int tile = job - (2 + role) * ntiles;
    float* pg = partial + (long long)tile * partial_stride(P.total);
    if (tid == 0) lt_prefetch_w1(S, timg, L);
    lt_biases(img, L, b1, b2, b3, tid);
    // the tile's samples (the same counter-RNG draws as the next-state jobs)
    if (tid < kLtRows) {
      const int i = tile * kLtRows + tid;
      rows_sh[tid] = i < batch ? (int)sample_entry(seed, tstep, i, rp) : -1;
    }
    __syncthreads();
    lt_load_x(xs, rp.s, rows_sh, L.n_in, L.k1, tid);
    lt_sync();
    ok = lt_forward(S, &bar_layer, player, tacc, timg, L, xs, h1s, h2s, b1, b2, tid, layer_out);
    if (!ok) break;
    // the tile's two next-state jobs (taken earlier by running CTAs, which
    // never wait) publish their Q-values; bounded wait
    if (tid == 0) {
      unsigned it = 0;
      while (qt_ld_acquire(sync + 1 + tile) < 2u && ++it < kQtWaitIters) __nanosleep(256);
      flag_sh = it < kQtWaitIters ? 1 : 0;
    }
    __syncthreads();
    if (!flag_sh) {
      ok = false;
      break;
    }
    // double-DQN targets y = r + gamma (1 - term) Q_target(s', argmax_a Q_online(s', a))
    if (tid < kLtRows) {
      const int i = tile * kLtRows + tid, e = rows_sh[tid];
      float y = 0.0f;
      if (e >= 0) {
        const float* qo = q2 + (long long)i * 5;
        const float* qt = q2 + ((long long)batch + i) * 5;
        int astar = 0;
        float best = __ldcg(qo);
        for (int a = 1; a < 5; ++a) {
          const float v = __ldcg(qo + a);
          if (v > best) {
            best = v;
            astar = a;
          }
        }
        const float nt = rp.term[e] ? 0.0f : 1.0f;
        y = rp.r[e] + gamma * nt * __ldcg(qt + astar);
        if (isnan(best)) y = best;  // a failed next-state job
      }
      y_sh[tid] = y;
    }
    __syncthreads();
    // dL/dQ(s, a) = clip(Q(s, a) - y) / B, back through the head's combine
    if (warp < 4) {
      const int r = warp * 32 + lane, e = rows_sh[r];
      float v[32];
      tmem_ld32(tacc + ((uint32_t)(warp * 32) << 16), v);
      float hl = 0.0f;
      float* dO = dout + r * kOutPad;
      for (int k = 0; k < kOutPad; ++k) dO[k] = 0.0f;
      if (e >= 0) {
        float o[kOut], qv[5];
#pragma unroll
        for (int j = 0; j < kOut; ++j) o[j] = v[j] + b3[j];
        greedy_action(o, qv, L.plain);
        int a = rp.a[e];
        float d;
        if (a >= 5) {
          atomicOr(fail, kTdFailAction);
          a = 0;
          d = __int_as_float(0x7fc00000);
        } else {
          d = qv[a] - y_sh[r];
        }
        const float ad = fabsf(d);
        hl = ad <= 1.0f ? 0.5f * d * d : ad - 0.5f;
        const float gq = (isnan(d) ? d : fminf(fmaxf(d, -1.0f), 1.0f)) / (float)batch;
        if (L.plain) {
          for (int k = 0; k < 5; ++k) dO[k] = k == a ? gq : 0.0f;
        } else {
          dO[0] = gq;
          for (int k = 0; k < 5; ++k) dO[1 + k] = (k == a ? gq : 0.0f) - gq / 5.0f;
        }
      }
      // the tile's Huber sum: lanes in order, then warps in order
      for (int off = 16; off > 0; off >>= 1) hl += __shfl_xor_sync(kFull, hl, off);
      if (lane == 0) hub_sh[warp] = hl;
    }
    lt_sync();
    // CUDA cores, thread per hidden unit n: dW3[o][n] = sum_s dO[s][o] H2[s][n],
    // dZ2[s][n] = (H2 > 0) sum_o dO[s][o] W3[o][n] written over H2 (BF16),
    // db2[n] = sum_s dZ2[s][n] (FP32)
    {
      const int n = tid;
      float w3c[kOut];
#pragma unroll
      for (int o = 0; o < kOut; ++o) w3c[o] = __bfloat162float(W3g[o * kLdh + n]);
      float acc3[kOut];
#pragma unroll
      for (int o = 0; o < kOut; ++o) acc3[o] = 0.0f;
      float db2 = 0.0f;
      // four rows at a time: their loads are independent of the stores
      for (int r0 = 0; r0 < kLtRows; r0 += 4) {
        bf16* hp[4];
        float h[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          hp[u] = reinterpret_cast<bf16*>(h2s + kmajor_offset(r0 + u, n, kLtRows));
          h[u] = __bfloat162float(*hp[u]);
        }
        bf16 z[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float* dO = dout + (r0 + u) * kOutPad;
          float dh = 0.0f;
#pragma unroll
          for (int o = 0; o < kOut; ++o) {
            acc3[o] += dO[o] * h[u];
            dh += dO[o] * w3c[o];
          }
          const float dz = h[u] > 0.0f ? dh : 0.0f;
          db2 += dz;
          z[u] = __float2bfloat16_rn(dz);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) *hp[u] = z[u];
      }
      if (role == 0) {
#pragma unroll
        for (int o = 0; o < kOut; ++o) pg[P.w3 + o * kHid + n] = acc3[o];
        pg[P.b2 + n] = db2;
        if (n < kOut) {
          float acc = 0.0f;
          for (int r = 0; r < kLtRows; ++r) acc += dout[r * kOutPad + n];
          pg[P.b3 + n] = acc;
        }
        if (n == 0) pg[P.total] = ((hub_sh[0] + hub_sh[1]) + hub_sh[2]) + hub_sh[3];
      }
    }
    fence_async_smem();
    lt_sync();
    if (role == 0) {
      // tensor cores: dW2 = dZ2^T H1 (M = out unit in two halves, N = in unit,
      // K = sample; both operands transposed) into columns [0, 512); the W2
      // quarters of dH1 stream in meanwhile
      if (tid == 0) {
        for (int h = 0; h < 2; ++h)
          lt_mma(tacc + 256u * h, smem_u32(h2s) + 16u * (uint32_t)h * kA, 128, kA, 2u * 128u, smem_u32(h1s), 128, kA,
                 2u * 128u, idesc_bf16_f32_t(kLtRows, kHid, 1, 1), kLtRows / 16, false);
        tc_commit(&bar_layer);
      }
      layer_out = true;
      ok = __syncthreads_and(mbar_wait(&bar_layer, player, kTcTries));
      player ^= 1u;
      layer_out = !ok;
      if (!ok) break;
      tc_fence_after();
      {
        // warp w: rows of lane quarter w % 4 (out unit 32 (w % 4) + lane of half
        // w / 4), 32 columns at a time through a 32 x 32 float tile of buffer 1
        // (rotated by the row: conflict-free both ways), then stored row by row
        // with the warp's 32 lanes on 32 consecutive columns (coalesced)
        const int quarter = warp & 3, h = warp >> 2, n0 = 128 * h + quarter * 32;
        float* st = reinterpret_cast<float*>(S.buf[1]) + warp * 32 * 32;
        for (int c = 0; c < kHid; c += 32) {
          float v[32];
          tmem_ld32(tacc + ((uint32_t)(quarter * 32) << 16) + 256u * h + (uint32_t)c, v);
#pragma unroll
          for (int k = 0; k < 32; ++k) st[lane * 32 + ((k + lane) & 31)] = v[k];
          __syncwarp();
#pragma unroll 8
          for (int r = 0; r < 32; ++r) pg[P.w2 + (long long)(n0 + r) * kHid + c + lane] = st[r * 32 + ((lane + r) & 31)];
          __syncwarp();
        }
      }
      fence_async_smem();  // the staging reads before buffer 1 takes a bulk copy
      lt_sync();
      continue;
    }  // role 0
    // dH1 = dZ2 W2^T (A = dZ2 K-major over the out unit, B = W2 quarters
    // transposed) into columns [0, 256)
    if (tid == 0) {
      for (int q = 0; q < 4; ++q) {
        const int b = q & 1;
        if (q < 2) S.load(b, timg + G.w2q + (uint32_t)q * w2q, w2q);
        if (q == 2) {
          S.load(0, timg + G.w2q + 2u * w2q, w2q);
          S.load(1, timg + G.w2q + 3u * w2q, w2q);
        }
        if (S.ready(b)) {
          lt_mma(tacc, smem_u32(h2s) + (uint32_t)(8 * q) * kA, kA, 128, 2u * kA, smem_u32(S.buf[b]), 128, 64u * 16u,
                 2u * 128u, idesc_bf16_f32_t(kLtRows, kHid, 0, 1), 64 / 16, q > 0);
          S.done(b);
        }
      }
      if (S.ok) tc_commit(&bar_layer);
    }
    layer_out = true;
    ok = __syncthreads_and(mbar_wait(&bar_layer, player, kTcTries));
    player ^= 1u;
    layer_out = !ok;
    if (!ok) break;
    tc_fence_after();
    {
      // dZ1 = (H1 > 0) dH1 written over H1 (BF16); db1 from the FP32 values
      const int quarter = warp & 3, r = quarter * 32 + lane, c0 = (warp >> 2) * 128;
      for (int c = c0; c < c0 + 128; c += 32) {
        float v[32];
        tmem_ld32(tacc + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint4* hp = reinterpret_cast<uint4*>(h1s + kmajor_offset(r, c + 8 * g, kLtRows));
          const uint4 hv = *hp;
          const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
          uint32_t w[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bool m0 = (hw[j] & 0xFFFFu) != 0u && !(hw[j] & 0x8000u);
            const bool m1 = (hw[j] >> 16) != 0u && !(hw[j] & 0x80000000u);
            v[8 * g + 2 * j] = m0 ? v[8 * g + 2 * j] : 0.0f;
            v[8 * g + 2 * j + 1] = m1 ? v[8 * g + 2 * j + 1] : 0.0f;
            w[j] = pack_bf16x2(v[8 * g + 2 * j], v[8 * g + 2 * j + 1]);
          }
          *hp = make_uint4(w[0], w[1], w[2], w[3]);
        }
        const float s = lt_colsum32(v, lane);
        red[quarter * kHid + c + lane] = s;
      }
    }
    fence_async_smem();
    lt_sync();
    if (tid < kHid) pg[P.b1 + tid] = ((red[tid] + red[kHid + tid]) + red[2 * kHid + tid]) + red[3 * kHid + tid];
    // dW1 = dZ1^T X (M = hidden unit in two halves, N = input feature,
    // K = sample; both operands transposed) into columns [0, 2 k1)
    if (tid == 0) {
      for (int h = 0; h < 2; ++h)
        lt_mma(tacc + (uint32_t)(h * L.k1), smem_u32(h1s) + 16u * (uint32_t)h * kA, 128, kA, 2u * 128u, smem_u32(xs),
               128, kA, 2u * 128u, idesc_bf16_f32_t(kLtRows, L.k1, 1, 1), kLtRows / 16, false);
      tc_commit(&bar_layer);
    }
    layer_out = true;
    ok = __syncthreads_and(mbar_wait(&bar_layer, player, kTcTries));
    player ^= 1u;
    layer_out = !ok;
    if (!ok) break;
    tc_fence_after();
    {
      // dW1 rows (hidden unit j, n_in inputs) staged over the dead H1 / H2
      // tiles with an odd row stride (conflict-free), then copied out: the
      // block is contiguous in the partial row (coalesced)
      const int quarter = warp & 3, h = warp >> 2, j = 128 * h + quarter * 32 + lane;
      const int sn = L.n_in | 1;
      float* st = reinterpret_cast<float*>(h1s);  // 256 x sn floats <= 70 KB of the 128 KB
      for (int c = 0; c < L.k1; c += 32) {
        float v[32];
        tmem_ld32(tacc + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(h * L.k1 + c), v);
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (c + k < L.n_in) st[j * sn + c + k] = v[k];
      }
      lt_sync();
      for (int t = tid; t < kHid * L.n_in; t += kLtThreads) pg[P.w1 + t] = st[(t / L.n_in) * sn + t % L.n_in];
    }
    lt_sync();  // the tile's buffers and tensor memory are reused by the next tile
  }
  if (!ok && tid == 0) atomicOr(fail, kTdFailCopy);
  if (tid == 0) {
    S.drain();
    if (layer_out) mbar_wait(&bar_layer, player, kTcTries);
  }
  lt_sync();
  if (warp == 0) tmem_free(tacc, 512);
}


// ------------------------------------------------------------- host side

namespace {
#define SG_CUDA(call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return sg_set_cuda_error(e_, #call); \
  } while (0)

size_t fwd_smem(const ImgLayout& L, int rows = kTile) {
  return (size_t)L.bytes + (size_t)rows * L.ld1 * 2 + 2ull * rows * kLdh * 2 + (size_t)rows * kOutPad * 4;
}
size_t grad_smem(const ImgLayout& L) {
  return (size_t)L.bytes + (size_t)kTile * L.ld1 * 2 + 3ull * kTile * kLdh * 2 + 2ull * kTile * kOutPad * 4;
}

int set_smem_attr(const void* fn, size_t bytes) {
  SG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return SG_OK;
}

// The online weights' copy in the tensor cores' layout follows every change
// of the online image (stream-ordered, so also inside captured graphs).
int refresh_tc_image(sg_qnet* q, cudaStream_t st) {
  k_tc_image<<<44, 256, 0, st>>>(q->img, q->IL, q->img_tc);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

int rebuild_image(sg_qnet* q, const float* th, uint8_t* img, cudaStream_t st) {
  const int n = image_elems(q->IL);
  k_build_image<<<(n + 255) / 256, 256, 0, st>>>(th, img, q->IL, q->PL);
  SG_CUDA(cudaGetLastError());
  if (img == q->img) return refresh_tc_image(q, st);
  // the target image's tensor-core copy (read by the tcgen05 learner)
  k_tc_image<<<44, 256, 0, st>>>(q->img_t, q->IL, q->img_tc_t);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

void free_qnet(sg_qnet* q) {
  if (!q) return;
  cudaFree(q->master);
  cudaFree(q->target);
  cudaFree(q->adam_m);
  cudaFree(q->adam_v);
  cudaFree(q->img);
  cudaFree(q->img_t);
  cudaFree(q->step);
  cudaFree(q->td_fail);
  cudaFree(q->partial);
  cudaFree(q->y);
  cudaFree(q->idx);
  cudaFree(q->img_tc);
  cudaFree(q->img_tc_t);
  cudaFree(q->q2);
  cudaFree(q->td_sync);
  delete q;
}
}  // namespace

#ifdef SG_DEBUG_BOUNDS
// This translation unit's debug bounds flag (read and cleared by sg_sim_status).
int sg_take_debug_bounds_qnet(unsigned* v) {
  unsigned z = 0;
  cudaError_t e = cudaMemcpyFromSymbol(v, g_debug_bounds, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_debug_bounds, &z, sizeof(unsigned));
  return e == cudaSuccess ? SG_OK : sg_set_cuda_error(e, "debug bounds flag");
}
#endif

extern "C" int sg_qnet_create(int32_t n_in, int32_t arch, int32_t max_batch, uint64_t seed, sg_qnet_t* out) {
  SG_RANGE("sg_qnet_create");
  if (!out || n_in < 1 || n_in > 69 || max_batch < 1 || max_batch > (1 << 16)) return SG_E_INVAL;
  if (arch != SG_QNET_DUELING && arch != SG_QNET_PAPER) return SG_E_INVAL;
  *out = nullptr;
  sg_qnet* q = new (std::nothrow) sg_qnet();
  if (!q) return SG_E_OOM;
  q->n_in = n_in;
  q->arch = arch;
  q->IL = img_layout(n_in, arch == SG_QNET_PAPER ? 1 : 0);
  q->PL = param_layout(n_in);
  q->max_batch = (max_batch + kTile - 1) / kTile * kTile;
  cudaGetDevice(&q->device);
  const size_t P = (size_t)q->PL.total;
  const size_t nblk = (size_t)q->max_batch / kTile;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  alloc((void**)&q->master, P * 4);
  alloc((void**)&q->target, P * 4);
  alloc((void**)&q->adam_m, P * 4);
  alloc((void**)&q->adam_v, P * 4);
  alloc((void**)&q->img, (size_t)q->IL.bytes);
  alloc((void**)&q->img_t, (size_t)q->IL.bytes);
  alloc((void**)&q->step, 8);
  alloc((void**)&q->td_fail, 4);
  alloc((void**)&q->partial, nblk * partial_stride(P) * 4);
  alloc((void**)&q->y, (size_t)q->max_batch * 4);
  alloc((void**)&q->idx, (size_t)q->max_batch * 4);
  alloc((void**)&q->img_tc, tc_img(q->IL.k1).bytes);
  alloc((void**)&q->img_tc_t, tc_img(q->IL.k1).bytes);
  alloc((void**)&q->q2, (size_t)2 * q->max_batch * 5 * 4);
  alloc((void**)&q->td_sync, (size_t)(1 + (q->max_batch + kLtRows - 1) / kLtRows) * 4);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&q->sms, cudaDevAttrMultiProcessorCount, q->device);
  if (e != cudaSuccess) {
    free_qnet(q);
    sg_set_cuda_error(e, "cudaMalloc");
    return SG_E_OOM;
  }
  int rc = SG_OK;
  if (e == cudaSuccess) e = cudaMemset(q->adam_m, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(q->adam_v, 0, P * 4);
  if (e == cudaSuccess) e = cudaMemset(q->step, 0, 8);
  if (e == cudaSuccess) e = cudaMemset(q->td_fail, 0, 4);
  if (e == cudaSuccess) e = cudaMemset(q->img, 0, (size_t)q->IL.bytes);
  if (e == cudaSuccess) e = cudaMemset(q->img_t, 0, (size_t)q->IL.bytes);
  if (e == cudaSuccess) {
    k_init_params<<<((int)P + 255) / 256, 256>>>(q->master, q->PL, n_in, q->IL.plain, seed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) rc = rebuild_image(q, q->master, q->img, 0);
  if (e == cudaSuccess && rc == SG_OK) e = cudaMemcpy(q->target, q->master, P * 4, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && rc == SG_OK) e = cudaMemcpy(q->img_t, q->img, (size_t)q->IL.bytes, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && rc == SG_OK)
    e = cudaMemcpy(q->img_tc_t, q->img_tc, tc_img(q->IL.k1).bytes, cudaMemcpyDeviceToDevice);
  if (e == cudaSuccess && rc == SG_OK) e = cudaDeviceSynchronize();
  if (e != cudaSuccess || rc != SG_OK) {
    free_qnet(q);
    return e != cudaSuccess ? sg_set_cuda_error(e, "sg_qnet_create") : rc;
  }
  // The limit is a property of the kernel, shared by every handle: set it for
  // the widest supported input so that a narrower network created later
  // cannot lower it below what a wider one launches with.
  const ImgLayout widest = img_layout(69);
  if ((rc = set_smem_attr((const void*)k_qnet_forward_tc, kTcSmemLaunch)) ||
      (rc = set_smem_attr((const void*)k_rollout_q_tc, qt_smem().bytes)) ||
      (rc = set_smem_attr((const void*)k_rollout_q<1, false>, fwd_smem(widest))) ||
      (rc = set_smem_attr((const void*)k_rollout_q<2, false>, fwd_smem(widest, 32))) ||
      (rc = set_smem_attr((const void*)k_rollout_q<1, true>, fwd_smem(widest))) ||
      (rc = set_smem_attr((const void*)k_rollout_q<2, true>, fwd_smem(widest, 32))) ||
      (rc = set_smem_attr((const void*)k_td_target, fwd_smem(widest))) ||
      (rc = set_smem_attr((const void*)k_td_grad, grad_smem(widest))) ||
      (rc = set_smem_attr((const void*)k_td_tc, kTcSmemLaunch))) {
    free_qnet(q);
    return rc;
  }
  *out = q;
  return SG_OK;
}

extern "C" int sg_qnet_destroy(sg_qnet_t q) {
  SG_RANGE("sg_qnet_destroy");
  if (!q) return SG_E_INVAL;
  cudaDeviceSynchronize();
  free_qnet(q);
  return SG_OK;
}

// The network's own (compact) parameter vector <-> the padded one the
// kernels use (identity for the dueling network).
static int64_t compact_params(const sg_qnet* q) { return q->IL.plain ? paper_params(q->n_in) : q->PL.total; }
static void to_padded(const sg_qnet* q, const float* compact, std::vector<float>& padded) {
  padded.assign((size_t)q->PL.total, 0.0f);
  for (int i = 0; i < q->PL.total; ++i) {
    const int j = q->IL.plain ? paper_index(i, q->PL, q->n_in) : i;
    if (j >= 0) padded[(size_t)i] = compact[j];
  }
}
static void to_compact(const sg_qnet* q, const std::vector<float>& padded, float* compact) {
  for (int i = 0; i < q->PL.total; ++i) {
    const int j = q->IL.plain ? paper_index(i, q->PL, q->n_in) : i;
    if (j >= 0) compact[j] = padded[(size_t)i];
  }
}
static int upload(const sg_qnet* q, float* dev, const float* host) {
  std::vector<float> v;
  to_padded(q, host, v);
  SG_CUDA(cudaMemcpy(dev, v.data(), v.size() * 4, cudaMemcpyHostToDevice));
  return SG_OK;
}
static int download(const sg_qnet* q, const float* dev, float* host) {
  std::vector<float> v((size_t)q->PL.total);
  SG_CUDA(cudaMemcpy(v.data(), dev, v.size() * 4, cudaMemcpyDeviceToHost));
  to_compact(q, v, host);
  return SG_OK;
}

extern "C" int sg_qnet_num_params(sg_qnet_t q, int64_t* n) {
  SG_RANGE("sg_qnet_num_params");
  if (!q || !n) return SG_E_INVAL;
  *n = compact_params(q);
  return SG_OK;
}

extern "C" int sg_qnet_set_params(sg_qnet_t q, const float* host, int64_t n, int32_t which) {
  SG_RANGE("sg_qnet_set_params");
  if (!q || !host || n != compact_params(q) || which < 0 || which > 2) return SG_E_INVAL;
  SG_CUDA(cudaDeviceSynchronize());
  if (which == 0 || which == 2) {
    int rc = upload(q, q->master, host);
    if (!rc) rc = rebuild_image(q, q->master, q->img, 0);
    if (rc) return rc;
  }
  if (which == 1 || which == 2) {
    int rc = upload(q, q->target, host);
    if (!rc) rc = rebuild_image(q, q->target, q->img_t, 0);
    if (rc) return rc;
  }
  SG_CUDA(cudaDeviceSynchronize());
  return SG_OK;
}

extern "C" int sg_qnet_get_params(sg_qnet_t q, float* host, int64_t n, int32_t which) {
  SG_RANGE("sg_qnet_get_params");
  if (!q || !host || n != compact_params(q) || which < 0 || which > 1) return SG_E_INVAL;
  SG_CUDA(cudaDeviceSynchronize());
  return download(q, which == 0 ? q->master : q->target, host);
}

extern "C" int sg_qnet_get_optimizer(sg_qnet_t q, float* m_host, float* v_host, int64_t n, uint64_t* steps) {
  SG_RANGE("sg_qnet_get_optimizer");
  if (!q || n != compact_params(q)) return SG_E_INVAL;
  SG_CUDA(cudaDeviceSynchronize());
  int rc = SG_OK;
  if (m_host) rc = download(q, q->adam_m, m_host);
  if (!rc && v_host) rc = download(q, q->adam_v, v_host);
  if (rc) return rc;
  if (steps) SG_CUDA(cudaMemcpy(steps, q->step, 8, cudaMemcpyDeviceToHost));
  return SG_OK;
}

extern "C" int sg_qnet_set_rollout_rows(sg_qnet_t q, int32_t rows) {
  SG_RANGE("sg_qnet_set_rollout_rows");
  if (!q || (rows != 0 && rows != 16 && rows != 32 && rows != 128)) return SG_E_INVAL;
  q->rollout_mt = rows / 16;
  return SG_OK;
}

extern "C" int sg_qnet_set_grid_limit(sg_qnet_t q, int32_t rollout_ctas, int32_t learner_ctas) {
  SG_RANGE("sg_qnet_set_grid_limit");
  if (!q || rollout_ctas < 0 || learner_ctas < 0) return SG_E_INVAL;
  q->lim_rollout = rollout_ctas;
  q->lim_learner = learner_ctas;
  return SG_OK;
}

extern "C" int sg_qnet_copy_params(sg_qnet_t dst, sg_qnet_t src, sg_stream_t stream) {
  SG_RANGE("sg_qnet_copy_params");
  if (!dst || !src || dst->n_in != src->n_in || dst->arch != src->arch) return SG_E_INVAL;
  const size_t P = (size_t)src->PL.total;
  SG_CUDA(cudaMemcpyAsync(dst->master, src->master, P * 4, cudaMemcpyDeviceToDevice, stream));
  SG_CUDA(cudaMemcpyAsync(dst->img, src->img, (size_t)src->IL.bytes, cudaMemcpyDeviceToDevice, stream));
  SG_CUDA(cudaMemcpyAsync(dst->img_tc, src->img_tc, tc_img(src->IL.k1).bytes, cudaMemcpyDeviceToDevice, stream));
  return SG_OK;
}

extern "C" int sg_qnet_set_optimizer(sg_qnet_t q, const float* m_host, const float* v_host, int64_t n,
                                     uint64_t steps) {
  SG_RANGE("sg_qnet_set_optimizer");
  if (!q || !m_host || !v_host || n != compact_params(q)) return SG_E_INVAL;
  SG_CUDA(cudaDeviceSynchronize());
  int rc = upload(q, q->adam_m, m_host);
  if (!rc) rc = upload(q, q->adam_v, v_host);
  if (rc) return rc;
  const unsigned long long st = steps;
  SG_CUDA(cudaMemcpy(q->step, &st, 8, cudaMemcpyHostToDevice));
  return SG_OK;
}

extern "C" int sg_qnet_forward(sg_qnet_t q, const float* obs_dev, int32_t M, float* q_dev, sg_stream_t stream) {
  SG_RANGE("sg_qnet_forward");
  if (!q || !obs_dev || !q_dev || M < 1) return SG_E_INVAL;
  // a persistent grid over the 128-row tiles
  const int ntiles = (M + kTcRows - 1) / kTcRows;
  k_qnet_forward_tc<<<std::min(ntiles, q->sms), kTfThreads, kTcSmemLaunch, stream>>>(q->img, q->img_tc, q->IL,
                                                                                     obs_dev, M, q_dev);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

extern "C" int sg_replay_create(int32_t slots_per_env, int32_t n_envs, int32_t obs_dim, int32_t reserve_slots,
                                sg_replay_t* out) {
  SG_RANGE("sg_replay_create");
  if (!out || slots_per_env < 1 || n_envs < 1 || obs_dim < 1) return SG_E_INVAL;
  if (reserve_slots < 0 || reserve_slots >= slots_per_env) return SG_E_INVAL;
  const long long cap = (long long)slots_per_env * n_envs;
  if (cap > (1ll << 31)) return SG_E_INVAL;
  *out = nullptr;
  sg_replay* r = new (std::nothrow) sg_replay();
  if (!r) return SG_E_OOM;
  r->cap = cap;
  cudaGetDevice(&r->device);
  r->d.slots = slots_per_env;
  r->d.n_envs = n_envs;
  r->d.obs_dim = obs_dim;
  r->d.reserve = reserve_slots;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  alloc((void**)&r->d.s, (size_t)cap * obs_dim * 4);
  alloc((void**)&r->d.s2, (size_t)cap * obs_dim * 4);
  alloc((void**)&r->d.a, (size_t)cap);
  alloc((void**)&r->d.r, (size_t)cap * 4);
  alloc((void**)&r->d.term, (size_t)cap);
  alloc((void**)&r->d.steps, 8);
  if (e == cudaSuccess) e = cudaMemset(r->d.steps, 0, 8);
  if (e != cudaSuccess) {
    cudaFree(r->d.s);
    cudaFree(r->d.s2);
    cudaFree(r->d.a);
    cudaFree(r->d.r);
    cudaFree(r->d.term);
    cudaFree(r->d.steps);
    delete r;
    sg_set_cuda_error(e, "cudaMalloc");
    return SG_E_OOM;
  }
  *out = r;
  return SG_OK;
}

extern "C" int sg_replay_destroy(sg_replay_t r) {
  SG_RANGE("sg_replay_destroy");
  if (!r) return SG_E_INVAL;
  cudaDeviceSynchronize();
  cudaFree(r->d.s);
  cudaFree(r->d.s2);
  cudaFree(r->d.a);
  cudaFree(r->d.r);
  cudaFree(r->d.term);
  cudaFree(r->d.steps);
  delete r;
  return SG_OK;
}

extern "C" int sg_replay_info(sg_replay_t r, int64_t* capacity, uint64_t* steps_recorded, void** s_dev, void** s2_dev,
                              void** a_dev, void** r_dev, void** term_dev) {
  SG_RANGE("sg_replay_info");
  if (!r) return SG_E_INVAL;
  if (capacity) *capacity = r->cap;
  if (steps_recorded) {
    SG_CUDA(cudaDeviceSynchronize());
    SG_CUDA(cudaMemcpy(steps_recorded, r->d.steps, 8, cudaMemcpyDeviceToHost));
  }
  if (s_dev) *s_dev = r->d.s;
  if (s2_dev) *s2_dev = r->d.s2;
  if (a_dev) *a_dev = r->d.a;
  if (r_dev) *r_dev = r->d.r;
  if (term_dev) *term_dev = r->d.term;
  return SG_OK;
}

extern "C" int sg_replay_read(sg_replay_t r, int64_t first, int64_t count, float* s_host, float* s2_host,
                              uint8_t* a_host, float* r_host, uint8_t* term_host) {
  SG_RANGE("sg_replay_read");
  if (!r || first < 0 || count < 0 || first + count > r->cap) return SG_E_INVAL;
  SG_CUDA(cudaDeviceSynchronize());
  const size_t od = (size_t)r->d.obs_dim;
  if (s_host) SG_CUDA(cudaMemcpy(s_host, r->d.s + first * od, count * od * 4, cudaMemcpyDeviceToHost));
  if (s2_host) SG_CUDA(cudaMemcpy(s2_host, r->d.s2 + first * od, count * od * 4, cudaMemcpyDeviceToHost));
  if (a_host) SG_CUDA(cudaMemcpy(a_host, r->d.a + first, count, cudaMemcpyDeviceToHost));
  if (r_host) SG_CUDA(cudaMemcpy(r_host, r->d.r + first, count * 4, cudaMemcpyDeviceToHost));
  if (term_host) SG_CUDA(cudaMemcpy(term_host, r->d.term + first, count, cudaMemcpyDeviceToHost));
  return SG_OK;
}

extern "C" int sg_replay_write(sg_replay_t r, int64_t first, int64_t count, const float* s_host, const float* s2_host,
                               const uint8_t* a_host, const float* r_host, const uint8_t* term_host,
                               uint64_t steps_recorded) {
  SG_RANGE("sg_replay_write");
  if (!r || first < 0 || count < 0 || first + count > r->cap) return SG_E_INVAL;
  if (count > 0 && (!s_host || !s2_host || !a_host || !r_host || !term_host)) return SG_E_INVAL;
  SG_CUDA(cudaDeviceSynchronize());
  const size_t od = (size_t)r->d.obs_dim;
  if (count > 0) {
    SG_CUDA(cudaMemcpy(r->d.s + first * od, s_host, count * od * 4, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(r->d.s2 + first * od, s2_host, count * od * 4, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(r->d.a + first, a_host, count, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(r->d.r + first, r_host, count * 4, cudaMemcpyHostToDevice));
    SG_CUDA(cudaMemcpy(r->d.term + first, term_host, count, cudaMemcpyHostToDevice));
  }
  const unsigned long long st = steps_recorded;
  SG_CUDA(cudaMemcpy(r->d.steps, &st, 8, cudaMemcpyHostToDevice));
  return SG_OK;
}

// VEM noise per env at T = n * t (t: env 0's step counter); see sg_vem_eps.
__global__ void k_vem_eps(const uint32_t* __restrict__ t_dev, int n, float e_min, float e_max, double or_start,
                          double or_final, double decay, float* __restrict__ eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double T = (double)n * (double)t_dev[0];
  const double frac = T / decay < 1.0 ? T / decay : 1.0;
  const double OR = or_start + (or_final - or_start) * frac;
  const double first = (double)n - OR;
  double e = (double)e_min;
  if ((double)i >= first) e = (double)e_min + (double)e_max * (((double)i - first) / (OR - 1.0));
  eps[i] = (float)e;
}

extern "C" int sg_vem_eps(sg_sim_t sim, float e_min, float e_max, double or_start, double or_final,
                          double decay_steps, float* eps_dev, sg_stream_t stream) {
  SG_RANGE("sg_vem_eps");
  if (!sim || !eps_dev) return SG_E_INVAL;
  const int n = sim->dc.n_envs;
  if (!(or_final >= 2.0 && or_final <= n && or_start >= 2.0 && or_start <= n && decay_steps > 0.0 &&
        e_min >= 0.0f && e_max >= 0.0f))
    return SG_E_INVAL;
  // u is [4][n]: ep_step, ep_id, t, fifo
  k_vem_eps<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(sim->ustate + 2 * (size_t)n, n, e_min, e_max, or_start,
                                                               or_final, decay_steps, eps_dev);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}

int sg_rollout_eps_q(sg_sim* sim, int K, sg_qnet* q, const float* eps, sg_replay* rp, float* obs, float* obs_seq,
                     uint8_t* act_seq, float* rew_seq, uint8_t* done_seq, cudaStream_t stream) {
  if (q->n_in != sim->dc.obs_dim) return SG_E_INVAL;
  ReplayDev rd;
  std::memset(&rd, 0, sizeof(rd));
  if (rp) {
    if (rp->d.n_envs != sim->dc.n_envs || rp->d.obs_dim != sim->dc.obs_dim) return SG_E_INVAL;
    rd = rp->d;
  }
  // 32 envs per CTA (two m-tiles) when that fills fewer waves than 16; the
  // shared-memory image limits a CTA to one per SM either way
  int sms = 0;
  SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sim->device));
  const int n = sim->dc.n_envs;
  const int waves16 = ((n + 15) / 16 + sms - 1) / sms, waves32 = ((n + 31) / 32 + sms - 1) / sms;
  // with dynamic obstacles the 32-env CTA (64 registers a thread) spills the
  // disc registers: 16 envs per CTA unless asked otherwise
  const bool dyn = sim->dc.n_dyn > 0;
  // 128 envs per CTA on the tcgen05 kernel when they fill every SM at least
  // once (or when asked for), without dynamic obstacles
  const bool tc = !dyn && (q->rollout_mt == 8 || (q->rollout_mt == 0 && n >= kQtEnvs * sms));
  const int mt = q->rollout_mt > 0 && q->rollout_mt <= 2 ? q->rollout_mt : (!dyn && waves32 < waves16 ? 2 : 1);
  if (tc) {
    // more than one wave of 128-env CTAs: slice the rollout into 4 to 6
    // segments over a resident grid so that no SM idles in a part-empty last
    // wave (the grid within the network's CTA cap, when one is set): the
    // count whose (block, segment) items fill the last round of the grid
    // best (65,536 envs: 5 segments, 429.7 M env-steps/s against 425.8 M
    // with 4, 427.0 M with 6, 413.5 M with 8)
    const int cap = q->lim_rollout > 0 ? std::min(q->lim_rollout, sms) : sms;
    const int nblk = (n + kQtEnvs - 1) / kQtEnvs;
    int seg = 0;
    if (nblk > cap && K >= 4) {
      double best = 0.0;
      for (int ns = 4; ns <= 6 && ns <= K; ++ns) {
        const int sl = (K + ns - 1) / ns;
        const long long items = (long long)nblk * ((K + sl - 1) / sl);
        const long long rounds = (items + cap - 1) / cap;
        const double fill = (double)items / ((double)rounds * cap);
        if (fill > best + 1e-9) {
          best = fill;
          seg = sl;
        }
      }
    }
    int grid = nblk;
    if (seg > 0) {
      grid = std::min(nblk * ((K + seg - 1) / seg), cap);
      SG_CUDA(cudaMemsetAsync(sim->q_sync_dev, 0, sizeof(unsigned) * (size_t)(nblk + 2), stream));
    }
    k_rollout_q_tc<<<grid, kQtThreads, qt_smem().bytes, stream>>>(
        sim->dc, sg_sim_ptrs(sim), q->img, q->img_tc, q->IL, K, eps, rd, rp ? 1 : 0, sim->map_order_dev, seg,
        seg > 0 ? sim->q_sync_dev : nullptr, obs, obs_seq, act_seq, rew_seq, done_seq);
  } else {
    // envs per CTA: the full tile, or fewer (down to half of it) when the
    // tiles would leave SMs idle (one CTA per SM: the staged image takes the
    // shared memory); 4,096 envs: 152 CTAs of 27 instead of 128 of 32
    const int rows = 16 * mt;
    const int epc = (n + rows - 1) / rows < sms ? std::max(rows / 2, (n + sms - 1) / sms) : rows;
    const int grid = (n + epc - 1) / epc;
    if (mt == 2)
      (dyn ? k_rollout_q<2, true> : k_rollout_q<2, false>)<<<grid, 1024, fwd_smem(q->IL, 32), stream>>>(
          sim->dc, sg_sim_ptrs(sim), q->img, q->IL, K, eps, rd, rp ? 1 : 0, sim->map_order_dev, epc, obs, obs_seq,
          act_seq, rew_seq, done_seq);
    else
      (dyn ? k_rollout_q<1, true> : k_rollout_q<1, false>)<<<grid, 512, fwd_smem(q->IL), stream>>>(
          sim->dc, sg_sim_ptrs(sim), q->img, q->IL, K, eps, rd, rp ? 1 : 0, sim->map_order_dev, epc, obs, obs_seq,
          act_seq, rew_seq, done_seq);
  }
  SG_CUDA(cudaGetLastError());
  if (rp) {
    k_replay_advance<<<1, 1, 0, stream>>>(rp->d.steps, K);
    SG_CUDA(cudaGetLastError());
  }
  return SG_OK;
}

extern "C" int sg_td_train_step(sg_qnet_t q, sg_replay_t rp, int32_t batch, float gamma, float lr,
                                int32_t target_every, uint64_t seed, float* loss_dev, float* grad_dev,
                                sg_stream_t stream) {
  SG_RANGE("sg_td_train_step");
  if (!q || !rp || batch < 1 || batch > q->max_batch || rp->d.obs_dim != q->n_in) return SG_E_INVAL;
  if (!(gamma >= 0.0f && gamma <= 1.0f) || !(lr >= 0.0f)) return SG_E_INVAL;
  SG_CUDA(cudaMemsetAsync(q->td_fail, 0, 4, stream));
  int nblk;
  if (batch >= kLtMinBatch) {
    // tcgen05 learner: 128-sample tiles, one partial gradient row per tile
    const int ntiles = (batch + kLtRows - 1) / kLtRows;
    nblk = ntiles;
    SG_CUDA(cudaMemsetAsync(q->td_sync, 0, (size_t)(1 + ntiles) * 4, stream));
    const int cap = q->lim_learner > 0 ? std::min(q->lim_learner, q->sms) : q->sms;
    k_td_tc<<<std::min(4 * ntiles, cap), kLtThreads, kTcSmemLaunch, stream>>>(
        q->img, q->img_t, q->img_tc, q->img_tc_t, q->IL, q->PL, rp->d, seed, q->step, batch, gamma, q->q2, q->idx,
        q->td_sync, q->partial, q->td_fail);
    SG_CUDA(cudaGetLastError());
  } else {
    // mma.sync learner: 16-sample tiles
    nblk = (batch + kTile - 1) / kTile;
    k_td_target<<<nblk, kThreads, fwd_smem(q->IL), stream>>>(q->img, q->img_t, q->IL, rp->d, seed, q->step, batch,
                                                              gamma, q->y, q->idx, q->td_fail);
    SG_CUDA(cudaGetLastError());
    k_td_grad<<<nblk, kThreads, grad_smem(q->IL), stream>>>(q->img, q->IL, q->PL, rp->d, q->idx, q->y, batch,
                                                            q->partial, q->td_fail);
    SG_CUDA(cudaGetLastError());
  }
  const int P = q->PL.total;
  k_adam<<<(P + 255) / 256, 256, 0, stream>>>(q->master, q->adam_m, q->adam_v, q->partial, nblk, q->PL, q->IL, q->img,
                                               q->step, lr, 0.9f, 0.999f, 1e-8f, loss_dev, grad_dev, batch,
                                               q->td_fail);
  SG_CUDA(cudaGetLastError());
  if (int rc = refresh_tc_image(q, stream)) return rc;
  if (lr > 0.0f) {
    k_step_advance<<<1, 1, 0, stream>>>(q->step, q->td_fail);
    SG_CUDA(cudaGetLastError());
    const int words = q->IL.bytes / 4;
    const int tc_words = (int)(tc_img(q->IL.k1).bytes / 4);
    const int n = std::max(P, std::max(words, tc_words));
    k_target_sync<<<(n + 255) / 256, 256, 0, stream>>>(q->step, target_every, q->master, q->target, q->img, q->img_t,
                                                        P, words, q->img_tc, q->img_tc_t, tc_words);
    SG_CUDA(cudaGetLastError());
  }
  return SG_OK;
}

// ------------------------------------------------------------------------
// TD loss and gradient without any allocation (sg_td_grad_noalloc).
//
// For callers that must not allocate device memory at all -- code running
// under a fixed memory budget, inside another framework's allocator, or in a
// context where cudaMalloc is not allowed -- and so cannot create a Q-network
// handle.  The caller passes the FP32 parameters and the batch; every
// intermediate buffer (BF16 weight images, TD targets, sample indices,
// per-CTA gradient partials) lives in one file-scope device array that each
// GPU holds from the moment the library is loaded until the process exits.
namespace {
constexpr int kNaMaxBatch = 256;
constexpr int kNaMaxIn = 69;
constexpr int kNaMaxBlk = kNaMaxBatch / kTile;
constexpr int kNaImgBytes = kHid * ((kNaMaxIn + 15) / 16 * 16 + 8) * 2 + kHid * kLdh * 2 + kOutPad * kLdh * 2 +
                            2 * kHid * 4 + kOutPad * 4;
constexpr int kNaImgSlot = (kNaImgBytes + 255) / 256 * 256;
// The widest image (69 inputs) is staged by the TD kernels in one mbarrier
// phase, whose transaction count holds at most 2^20 - 1 bytes.
static_assert(kNaImgBytes + 16 < (1 << 20), "one weight image fits an mbarrier phase's transaction count");
constexpr int kNaMaxParams = kHid * kNaMaxIn + kHid + kHid * kHid + kHid + kOut * kHid + kOut;
constexpr long long kNaOffY = 2ll * kNaImgSlot;
constexpr long long kNaOffIdx = kNaOffY + kNaMaxBatch * 4;
constexpr long long kNaOffFail = kNaOffIdx + kNaMaxBatch * 4;
constexpr long long kNaOffPartial = (kNaOffFail + 4 + 255) / 256 * 256;
constexpr long long kNaBytes = kNaOffPartial + (long long)kNaMaxBlk * partial_stride(kNaMaxParams) * 4;
}  // namespace

static __device__ __align__(256) unsigned char g_td_noalloc_scratch[kNaBytes];

// Double-DQN targets for an explicit batch (sample i is row i).
__global__ void __launch_bounds__(kThreads, 1)
    k_td_target_given(const uint8_t* __restrict__ img, const uint8_t* __restrict__ img_t, ImgLayout L, ReplayDev b,
                      int batch, float gamma, float* __restrict__ y, int* __restrict__ idx) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* sw = smem;
  bf16* X = reinterpret_cast<bf16*>(smem + L.bytes);
  bf16* H1 = X + kTile * L.ld1;
  bf16* H2 = H1 + kTile * kLdh;
  float* O = reinterpret_cast<float*>(H2 + kTile * kLdh);
  __shared__ int rows[kTile];
  __shared__ int astar[kTile];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * kTile + warp;
  if (lane == 0) {
    rows[warp] = i < batch ? i : -1;
    if (i < batch) idx[i] = i;
  }
  stage_image(sw, img, L.bytes);
  __syncthreads();
  gather_tile(X, L.ld1, b.s2, rows, b.obs_dim, warp, lane);
  __syncthreads();
  mlp_tile(qw_at(sw, L), X, H1, H2, O, warp, lane);
  if (lane == 0) astar[warp] = (int)greedy_action(O + warp * kOutPad, nullptr, L.plain);
  __syncthreads();
  stage_image(sw, img_t, L.bytes);
  __syncthreads();
  mlp_tile(qw_at(sw, L), X, H1, H2, O, warp, lane);
  if (lane == 0 && i < batch) {
    float qv[5];
    greedy_action(O + warp * kOutPad, qv, L.plain);
    const float nt = b.term[i] ? 0.0f : 1.0f;
    y[i] = b.r[i] + gamma * nt * qv[astar[warp]];
  }
}

namespace {
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[kNaMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (in host code its name is only a host-side stand-in) and
// the shared-memory limits of the kernels this path launches.
int na_setup(unsigned char** out) {
  int dev = 0;
  SG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return sg_set_error_text("sg_td_grad_noalloc: device ordinal too large", SG_E_INVAL);
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    SG_CUDA(cudaGetSymbolAddress(&p, g_td_noalloc_scratch));
    const ImgLayout L = img_layout(kNaMaxIn);
    int rc = set_smem_attr((const void*)k_td_target_given, fwd_smem(L));
    if (!rc) rc = set_smem_attr((const void*)k_td_grad, grad_smem(L));
    if (rc) return rc;
    g_na_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_ptr[dev];
  return SG_OK;
}
}  // namespace

extern "C" int sg_td_grad_noalloc(const float* params_dev, const float* target_params_dev, int32_t n_in,
                                  const float* s_dev, const uint8_t* a_dev, const float* r_dev, const float* s2_dev,
                                  const uint8_t* term_dev, int32_t batch, float gamma, float* loss_dev,
                                  float* grad_dev, sg_stream_t stream) {
  SG_RANGE("sg_td_grad_noalloc");
  if (!params_dev || !target_params_dev || !s_dev || !a_dev || !r_dev || !s2_dev || !term_dev || !grad_dev)
    return sg_set_error_text("sg_td_grad_noalloc: a required pointer is NULL", SG_E_INVAL);
  if (n_in < 1 || n_in > kNaMaxIn)
    return sg_set_error_text("sg_td_grad_noalloc: n_in must be in [1, 69] (static scratch limit)", SG_E_INVAL);
  if (batch < 1 || batch > kNaMaxBatch)
    return sg_set_error_text("sg_td_grad_noalloc: batch must be in [1, 256] (static scratch limit)", SG_E_INVAL);
  if (!(gamma >= 0.0f && gamma <= 1.0f)) return sg_set_error_text("sg_td_grad_noalloc: gamma outside [0, 1]", SG_E_INVAL);
  unsigned char* base = nullptr;
  int rc = na_setup(&base);
  if (rc) return rc;
  const ImgLayout IL = img_layout(n_in);
  const ParamLayout PL = param_layout(n_in);
  uint8_t* img = base;
  uint8_t* img_t = base + kNaImgSlot;
  float* y = reinterpret_cast<float*>(base + kNaOffY);
  int* idx = reinterpret_cast<int*>(base + kNaOffIdx);
  float* partial = reinterpret_cast<float*>(base + kNaOffPartial);
  unsigned* fail = reinterpret_cast<unsigned*>(base + kNaOffFail);
  ReplayDev b;
  std::memset(&b, 0, sizeof(b));
  b.s = const_cast<float*>(s_dev);
  b.s2 = const_cast<float*>(s2_dev);
  b.a = const_cast<uint8_t*>(a_dev);
  b.r = const_cast<float*>(r_dev);
  b.term = const_cast<uint8_t*>(term_dev);
  b.slots = 1;
  b.n_envs = batch;
  b.obs_dim = n_in;
  const int ne = image_elems(IL);
  k_build_image<<<(ne + 255) / 256, 256, 0, stream>>>(params_dev, img, IL, PL);
  SG_CUDA(cudaGetLastError());
  k_build_image<<<(ne + 255) / 256, 256, 0, stream>>>(target_params_dev, img_t, IL, PL);
  SG_CUDA(cudaGetLastError());
  const int nblk = (batch + kTile - 1) / kTile;
  SG_CUDA(cudaMemsetAsync(fail, 0, 4, stream));
  k_td_target_given<<<nblk, kThreads, fwd_smem(IL), stream>>>(img, img_t, IL, b, batch, gamma, y, idx);
  SG_CUDA(cudaGetLastError());
  k_td_grad<<<nblk, kThreads, grad_smem(IL), stream>>>(img, IL, PL, b, idx, y, batch, partial, fail);
  SG_CUDA(cudaGetLastError());
  k_adam<<<(PL.total + 255) / 256, 256, 0, stream>>>(nullptr, nullptr, nullptr, partial, nblk, PL, IL, nullptr,
                                                      nullptr, 0.0f, 0.9f, 0.999f, 1e-8f, loss_dev, grad_dev, batch,
                                                      fail);
  SG_CUDA(cudaGetLastError());
  return SG_OK;
}
