// The consumer kernels of depth 4, all tile sizes (see k_explain.cuh).
#include "k_explain.cuh"

namespace wdf {
WDF_EXPLAIN_DEPTH(4, )
}  // namespace wdf
