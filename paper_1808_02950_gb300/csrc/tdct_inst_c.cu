// Instantiations of the fused codec for r-classes group C (see tdct_classes.h).
#include "tdct_classes.h"
#include "tdct_kernels.cuh"

namespace tdct {
#define TDCT_INST(R)                                                                      \
  template cudaError_t launch_codec<R, 0>(const PlaneTable&, const CodecParams&,          \
                                          unsigned long long*, int, cudaStream_t);        \
  template cudaError_t launch_codec<R, 1>(const PlaneTable&, const CodecParams&,          \
                                          unsigned long long*, int, cudaStream_t);
TDCT_FOR_EACH_CLASS_C(TDCT_INST)
#undef TDCT_INST
}  // namespace tdct
