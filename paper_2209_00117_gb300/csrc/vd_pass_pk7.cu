// vd_pass_pk7.cu -- the position-tagged dJFA passes of layout M = 7
// (32768 to 2^17 - 1 seeds, window +-64); one translation unit per layout so that they compile in
// parallel.
#include "vd_pass_pk.cuh"

namespace vdi {
template int launch_pass_pk_m<7>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t, bool);
}  // namespace vdi
