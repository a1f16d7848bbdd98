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
  size_t arena_bytes = 0;
  size_t smem = 0;
  int dtype = -1;
};

// Validate requests and build descriptors + work table (no device work).
fs_status plan_requests(const fs_request *reqs, int n, BatchPlan *bp);

}  // namespace fs
