// sg_host.h -- host-side objects behind the C handles (internal).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "sg_device.cuh"
#include "sparrow_gb.h"

struct sg_sim {
  sg_sim_config cfg;
  sg::DevCfg dc;
  int n_maps = 0;
  int device = 0;
  int step_epw = 0;  // envs per warp of k_step (0 = not chosen yet)
  long long atlas_words = 0;
  long long clr_bytes = 0;
  std::vector<sg::MapDesc> maps_host;
  uint32_t* atlas = nullptr;
  uint8_t* clr = nullptr;
  uint8_t* sec = nullptr;      // sector skip planes (dc.n_sec > 1), else null
  long long sec_bytes = 0;
  sg::MapDesc* maps_dev = nullptr;
  int* env_map_dev = nullptr;
  int* env_beams_dev = nullptr;
  float* fstate = nullptr;     // [9][n]
  uint32_t* ustate = nullptr;  // [4][n]
  float* dyn = nullptr;        // [4 n_dyn][n] dynamic obstacles (null when n_dyn = 0)
  uint32_t* status_dev = nullptr;
  // launch configuration of the random rollout (sg_sim_set_launch)
  sg_launch launch = {SG_ROLLOUT_GRID, 4, 1, 0, 0, 0, 0, 0};  // no slicing, default wait bound
  int persistent_blocks = 0;
  int* order_dev = nullptr;      // work list (cost-sorted env indices) or null
  int* map_order_dev = nullptr;  // env indices grouped by map (stable), for per-CTA map locality
  unsigned* queue_dev = nullptr; // work-list cursor of the persistent kernel
  unsigned* pipe_sync_dev = nullptr;  // time-sliced pipelined rollout: segment flags, item counter, abort word
  size_t pipe_sync_words = 0;
  unsigned* q_sync_dev = nullptr;  // time-sliced fused Q rollout: per-block segment flags, item counter, abort word
};

// An NVTX range over the body of a C entry point (named after it), so that
// a timeline tool shows each library call; free when no tool is attached.
struct SgRange {
  explicit SgRange(const char* name) { nvtxRangePushA(name); }
  ~SgRange() { nvtxRangePop(); }
  SgRange(const SgRange&) = delete;
  SgRange& operator=(const SgRange&) = delete;
};
#define SG_RANGE(name) SgRange sg_range_(name)

sg::SimPtrs sg_sim_ptrs(sg_sim* s);
long long sg_state_bytes(const sg_sim* s);
int sg_set_cuda_error(cudaError_t e, const char* what);
int sg_set_error_text(const char* msg, int code);
