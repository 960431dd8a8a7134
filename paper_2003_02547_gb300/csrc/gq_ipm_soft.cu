// The block kernel with the slack elimination of soft constraints (Sec. 2.2)
// compiled in; launched by the host for batches whose block bucket holds QPs
// with slacks.  The shared-memory planner keeps one external definition (in
// gq_ipm.cu): this unit's copy is renamed.
#define GQ_IPM_SOFT 1
#define smem_plan smem_plan_soft
#include "gq_ipm.cu"
