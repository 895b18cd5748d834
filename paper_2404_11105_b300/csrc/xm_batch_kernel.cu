// The batched matcher (k_match_batch, launch_batch) in a translation unit of
// its own. ptxas of CUDA 13.0 crashes on a unit that holds both the
// batched kernel's leaf-product walk and the k_match instantiations, so
// this file compiles the matcher source with XM_BATCH_TU set, which keeps
// the device helpers and the batched kernel and leaves out the rest.
#define XM_BATCH_TU 1
#include "xm_kernels.cu"
