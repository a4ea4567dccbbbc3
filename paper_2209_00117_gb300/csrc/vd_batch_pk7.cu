// vd_batch_pk7.cu -- the batched engine's round kernel on position-tagged
// words of layout M = 7 (vd_batch_pk.cuh); one translation unit per layout.
#include "vd_batch_pk.cuh"

namespace vdb {
template int launch_round_pk_m<7>(const BatchArgs&, int, int, int, cudaStream_t);
}  // namespace vdb
