// vd_pass_pk4.cu -- the position-tagged dJFA passes of layout M = 4
// (2^18 + 1 to 2^22 seeds, window +-8, the label split around the x field);
// one translation unit per layout so that they compile in parallel.
#include "vd_pass_pk.cuh"

namespace vdi {
template int launch_pass_pk_m<4>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t, bool);
}  // namespace vdi
