// Instantiations of the launchers for int32 column indices.
#include "launch.cuh"
namespace sg {
SG_INSTANTIATE_IT(int32_t)
}
