// The block kernel with the tensor-core (tcgen05) stage products of the FP32
// factor compiled in; launched by the host for mixed-precision batches whose
// block bucket has large stages (128 <= nu + nx <= 256, nx <= 128, no
// general rows) when the schedule allows tensor cores.  Kept apart from the
// other variants because compiling the tensor-core path into one kernel
// changes its register allocation for every batch (measured: ragged batches
// 1.7x slower).  The shared-memory planner of this unit is renamed.
#define GQ_IPM_TC 1
#define smem_plan smem_plan_tc
#include "gq_ipm.cu"
