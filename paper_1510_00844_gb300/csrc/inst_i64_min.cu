// Instantiations of the numeric launchers for the (min, +) and
// (min, select2nd) semirings, int64_t column indices.
#include "launch.cuh"
namespace sg {
SG_INSTANTIATE_IT_V(int64_t, MinPlus<double>)
SG_INSTANTIATE_IT_V(int64_t, MinPlus<int64_t>)
SG_INSTANTIATE_IT_V(int64_t, MinSel<double>)
SG_INSTANTIATE_IT_V(int64_t, MinSel<int64_t>)
}
