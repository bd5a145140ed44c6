// The consumer kernels of depth 2, all tile sizes (see k_explain.cuh).
#include "k_explain.cuh"

namespace wdf {
WDF_EXPLAIN_DEPTH(2, )
}  // namespace wdf
