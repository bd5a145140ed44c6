// The consumer kernels of depth 5, all tile sizes (see k_explain.cuh).
#include "k_explain.cuh"

namespace wdf {
WDF_EXPLAIN_DEPTH(5, )
}  // namespace wdf
