// Instantiations of the generic-T codec for r-classes group B (tdct_generic_impl.cuh).
#include "tdct_generic_impl.cuh"

namespace tdct {
#define TDCT_GEN_INST(R)                                                                      \
  template cudaError_t launch_codec_generic<R, 0>(const PlaneTable&, const GenericParams&,    \
                                                  unsigned long long*, cudaStream_t);         \
  template cudaError_t launch_codec_generic<R, 1>(const PlaneTable&, const GenericParams&,    \
                                                  unsigned long long*, cudaStream_t);
TDCT_FOR_EACH_CLASS_B(TDCT_GEN_INST)
#undef TDCT_GEN_INST

}  // namespace tdct
