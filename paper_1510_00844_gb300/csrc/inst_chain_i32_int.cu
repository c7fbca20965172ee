// Persistent chain kernels, int32_t column indices, int64_t and NoVal values (one
// unit per pair, so that they compile in parallel with the other units).
#include "chain_launch.h"

namespace sg {
SG_INSTANTIATE_CHAIN(int32_t, int64_t, kChainThreads)
SG_INSTANTIATE_CHAIN(int32_t, NoVal, kChainThreads)
}  // namespace sg
