// The consumer kernels of depth 8, 32 rows per tile (see k_explain.cuh).
#include "k_explain.cuh"

namespace wdf {
WDF_EXPLAIN_TILE(8, 32, )
}  // namespace wdf
