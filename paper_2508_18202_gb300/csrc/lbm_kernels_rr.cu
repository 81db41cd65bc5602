// lbm_kernels_rr.cu -- the stream-collide kernels of lbm_kernels.cu compiled
// with the recursive regularized collision (third-order D3Q19 equilibrium,
// arXiv:2508.18202 Sec. 2.2) in place of BGK.  The step launchers land in
// namespace sclbm::rr.
#define SCLBM_RR_UNIT 1
#include "lbm_kernels.cu"
