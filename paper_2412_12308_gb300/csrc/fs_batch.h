// fs_batch.h -- batch planning shared by the batch executor and the server.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "fs_host.h"

namespace fs {

struct BatchPlan {
  std::vector<Desc> descs;       // in execution (largest-first) order
  std::vector<int> req_of_desc;  // request index of each desc
  std::vector<size_t> ws_off;    // arena offset of each desc's workspace
  std::vector<int4> units;       // work table: (desc, kind, index, field)
  std::vector<char> direct;      // desc runs as standalone pass kernels, not units
  size_t arena_bytes = 0;
  size_t smem = 0;
  int dtype = -1;
  int threads = 512;             // batch CTA size: 256 when every unit fits (two CTAs per SM)
  // single-CTA small problems of a batch that also has work units: their
  // units are the last n_small_units of the table and run as a second,
  // concurrent launch of small_threads-thread CTAs with small_smem bytes
  int n_small_units = 0;
  int small_threads = 512;
  size_t small_smem = 0;
};

// Validate requests and build descriptors + work table (no device work).
// keep_out[i] (optional): device buffer that receives request i's forward
// half spectrum (diffusion / wave solves with zero initial velocity).
// direct_min_points > 0: problems with nx*ny >= it run as standalone pass
// kernels (before the persistent launch) instead of work units.
fs_status plan_requests(const fs_request *reqs, int n, BatchPlan *bp, void *const *keep_out = nullptr,
                        long long direct_min_points = 0);

// Submit a planned batch on `stream` (see fs_batch_submit).
// ext_arena (optional, >= the batch's workspace bytes) replaces the slot's own
// arena; *ws_bytes_out (optional) receives the batch's workspace bytes.
fs_status batch_submit_internal(const fs_request *reqs, int n, void *const *keep_out, uint64_t *ticket_out,
                                cudaStream_t stream, char *ext_arena = nullptr, size_t ext_bytes = 0,
                                long long direct_min_points = 0);

// Workspace bytes one request needs in a batch arena (validates it).
fs_status request_workspace(const fs_request &r, size_t *bytes);

}  // namespace fs
