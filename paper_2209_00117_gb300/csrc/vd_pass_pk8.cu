// vd_pass_pk8.cu -- the position-tagged dJFA passes of layout M = 8
// (up to 32767 seeds, window +-128); one translation unit per layout so that they compile in
// parallel.
#include "vd_pass_pk.cuh"

namespace vdi {
// layouts 4, 6 and 7 are instantiated in their own translation units
extern template int launch_pass_pk_m<4>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t,
                                         bool);
extern template int launch_pass_pk_m<6>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t,
                                         bool);
extern template int launch_pass_pk_m<7>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t,
                                         bool);
template int launch_pass_pk_m<8>(const vdk::PassArgs&, dim3, dim3, int32_t, int, int, bool, cudaStream_t, bool);

int pk_bits(int32_t n) {
  // the label code 2^lb - 1 marks an empty pixel: below it for M = 7 and 8;
  // M = 6 and 4 carry a separate empty bit and so take up to 2^18 and 2^22
  // labels.  (M = 7 below 2^16 seeds: the frame's first pass folds with the
  // narrow byte-offset key, whose 16-bit label field the word bits then
  // follow.)
  if (n >= 1 && n <= 32767) return 8;
  if (n >= 32768 && n <= 131071) return 7;
  if (n >= 131072 && n <= 262144) return 6;
  if (n > 262144 && n <= (1 << 22)) return 4;
  return 0;
}

int launch_pass_pk(const vdk::PassArgs& a, dim3 grid, dim3 block, int32_t nb, int m, int ksel, int mode,
                   bool dedup, cudaStream_t st, bool pdl) {
  if (ksel > 2 || mode < 0 || mode > 2) return vd_fail(VD_EINVAL, "packed pass: step %d, mode %d", a.k, mode);
  switch (m) {
    case 4: return launch_pass_pk_m<4>(a, grid, block, nb, ksel, mode, dedup, st, pdl);
    case 6: return launch_pass_pk_m<6>(a, grid, block, nb, ksel, mode, dedup, st, pdl);
    case 7: return launch_pass_pk_m<7>(a, grid, block, nb, ksel, mode, dedup, st, pdl);
    case 8: return launch_pass_pk_m<8>(a, grid, block, nb, ksel, mode, dedup, st, pdl);
    default: return vd_fail(VD_EINVAL, "packed pass: layout %d", m);
  }
}
}  // namespace vdi
