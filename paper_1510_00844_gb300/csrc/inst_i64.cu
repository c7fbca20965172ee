// Instantiations of the launchers for int64 column indices.
#include "launch.cuh"
namespace sg {
SG_INSTANTIATE_IT(int64_t)
}
