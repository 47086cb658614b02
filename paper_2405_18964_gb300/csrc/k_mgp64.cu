// k_mgp64.cu -- the FP64 instantiation of the velocity multigrid with
// compile-time level sizes (k_mgp.cu), compiled as a translation unit of its
// own so that the build runs the two instantiations in parallel.
#define PINT_MGP_FP64
#include "k_mgp.cu"
