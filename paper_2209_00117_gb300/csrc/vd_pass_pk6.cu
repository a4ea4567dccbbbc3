// vd_pass_pk6.cu -- the position-tagged dJFA passes of layout M = 6
// (2^17 to 2^18 seeds, window +-32); one translation unit per layout so that they compile in
// parallel.
#include "vd_pass_pk.cuh"

namespace vdi {
template int launch_pass_pk_m<6>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t, bool);
}  // namespace vdi
