// The batch handle (host memory owned by the caller): planner output shared
// by the setters, the transfers, the solve entry points and the server.
#pragma once

#include <cstdint>

#include "gq_internal.h"
#include "gq_launch.h"

namespace gq {

struct SlotEntry {
  int64_t key;    // slot id, -1 = empty
  int64_t block;  // data offset (doubles)
  int32_t stage;  // first stage using this slot
  int32_t pad;
};

// Records a per-thread error message (read back by gq_last_error) and
// returns `code`.
int set_error(int code, const char* fmt, ...);

}  // namespace gq

struct gq_batch {
  uint32_t magic;
  int32_t nqp;
  int64_t n_stages, n_slots, hash_cap;
  gq::Layout L;
  gq_sizes sizes;
  int32_t ngmax;
  int32_t nwarp;        // QPs run one per warp; they lead the order array
  int32_t soft_block;   // 1: some QP of the block bucket has slacks (launch the soft kernel variant)
  int32_t warp_max_nv;  // schedule: largest nu + nx (and nx) of a QP run one per warp
  int32_t block_threads;  // schedule: threads per block of the block kernel
  int32_t tensor_cores;   // schedule: tcgen05 products for large FP32 stages
  gq::Shape shape_w, shape_b;
  gq::QpDesc* qp;
  gq::StageDesc* st;
  int32_t* order;
  int32_t* slot_stage;  // first stage of every distinct data block
  gq::SlotEntry* hash;
  void *host_in, *host_sol, *dev_in, *dev_sol, *dev_ws;
};
