// The consumer kernels of depth 7, all tile sizes (see k_explain.cuh).
#include "k_explain.cuh"

namespace wdf {
WDF_EXPLAIN_DEPTH(7, )
}  // namespace wdf
