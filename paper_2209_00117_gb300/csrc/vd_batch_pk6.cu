// vd_batch_pk6.cu -- the batched engine's round kernel on position-tagged
// words of layout M = 6 (vd_batch_pk.cuh); one translation unit per layout.
#include "vd_batch_pk.cuh"

namespace vdb {
template int launch_round_pk_m<6>(const BatchArgs&, int, int, int, cudaStream_t);
}  // namespace vdb
