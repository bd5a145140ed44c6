// The consumer kernels of depth 3, all tile sizes (see k_explain.cuh).
#include "k_explain.cuh"

namespace wdf {
WDF_EXPLAIN_DEPTH(3, )
}  // namespace wdf
