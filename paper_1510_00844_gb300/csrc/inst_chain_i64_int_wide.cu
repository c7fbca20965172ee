// Persistent chain kernels with 1024-thread blocks, int64_t column indices,
// int64_t and NoVal values (one unit per pair, so that they compile in
// parallel with the other units).
#include "chain_launch.h"

namespace sg {
SG_INSTANTIATE_CHAIN(int64_t, int64_t, kChainThreadsWide)
SG_INSTANTIATE_CHAIN(int64_t, NoVal, kChainThreadsWide)
}  // namespace sg
