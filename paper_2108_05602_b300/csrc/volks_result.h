// The opaque volks_result of include/volks.h: a view of one segment's
// search (owned by the handle for volks_search_segment, borrowed from the
// plan for volks_plan_result).
#pragma once
#include <vector>

#include <cuda_runtime.h>

#include "../../include/volks.h"
#include "volks_job.h"

struct volks_result {
  vk::SegJob* job = nullptr;          // the segment's state
  volks_plan* plan = nullptr;         // plan results: the owning plan
  vk::SegJob* own_job = nullptr;      // non-null when this handle owns it
  bool borrowed = false;              // plan results: volks_free is a no-op
  cudaStream_t stream = nullptr;      // stream of the last launch touching it
  cudaEvent_t ev[6] = {};
  unsigned long long* counter = nullptr;
  unsigned int* d_err = nullptr;      // tensor-core search: bounded-wait error flag
  int n_launch = 0, n_search_launch = 0;
  bool synced = false, have_cands = false;
  std::vector<volks_candidate> cands;
};

// Stage times of a plan's last run.
int vk_plan_timing(volks_plan* p, volks_timing* t);

// Re-run the window match of a single-chunk job into its (regrown)
// candidate buffer on r->stream.
int vk_rerun_match(volks_result* r);

// Wait for the result's stream and check the tensor-core error flag.
int vk_sync_result(volks_result* r);
