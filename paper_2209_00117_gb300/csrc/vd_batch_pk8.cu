// vd_batch_pk8.cu -- the batched engine's round kernel on position-tagged
// words of layout M = 8 (vd_batch_pk.cuh); one translation unit per layout.
#include "vd_batch_pk.cuh"

namespace vdb {
template int launch_round_pk_m<8>(const BatchArgs&, int, int, int, cudaStream_t);
extern template int launch_round_pk_m<6>(const BatchArgs&, int, int, int, cudaStream_t);
extern template int launch_round_pk_m<7>(const BatchArgs&, int, int, int, cudaStream_t);

int launch_round_pk(int m, const BatchArgs& A, int r, int t0, int n_tiles, cudaStream_t st) {
  switch (m) {
    case 6: return launch_round_pk_m<6>(A, r, t0, n_tiles, st);
    case 7: return launch_round_pk_m<7>(A, r, t0, n_tiles, st);
    case 8: return launch_round_pk_m<8>(A, r, t0, n_tiles, st);
    default: return vd_fail(VD_EINVAL, "batched packed round: layout %d", m);
  }
}
}  // namespace vdb
