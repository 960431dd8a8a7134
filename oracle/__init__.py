"""CPU FP64 oracle (test infrastructure only; see ocp_ipm)."""
