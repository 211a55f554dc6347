// Instantiations of the u8 FP32 exact-DCT kernels for some r-classes (tdct_dct.cuh).
#include "tdct_classes.h"
#include "tdct_dct.cuh"

namespace tdct {
#define TDCT_DCT_INST(R)                                                                  \
  template cudaError_t launch_dct<R, 0, false, false>(                                    \
      const PlaneDesc&, const DctParams&, float*, unsigned long long*, cudaStream_t, int);
TDCT_FOR_EACH_CLASS_A(TDCT_DCT_INST) TDCT_FOR_EACH_CLASS_B(TDCT_DCT_INST)
#undef TDCT_DCT_INST
}  // namespace tdct
