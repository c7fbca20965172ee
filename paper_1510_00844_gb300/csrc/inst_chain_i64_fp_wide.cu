// Persistent chain kernels with 1024-thread blocks, int64_t column indices,
// double and float values (one unit per pair, so that they compile in
// parallel with the other units).
#include "chain_launch.h"

namespace sg {
SG_INSTANTIATE_CHAIN(int64_t, double, kChainThreadsWide)
SG_INSTANTIATE_CHAIN(int64_t, float, kChainThreadsWide)
}  // namespace sg
