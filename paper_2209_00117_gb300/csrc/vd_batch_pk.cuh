// vd_batch_pk.cuh -- the batched engine's passes on position-tagged words.
//
// In the launch-per-round mode a simulation's last dJFA passes may run on
// position-tagged words (the single-simulation passes of vd_pass_pk.cuh, each
// simulation with its own word layout M: 8 up to 32767 seeds, 7 up to
// 2^17 - 1, 6 up to 2^18).  The plan puts, in every round, the tiles of such
// simulations first, grouped by M, and each group runs in the kernel of its
// layout below, one translation unit per layout (vd_batch_pk<M>.cu), so that
// they compile in parallel and keep their own register budget (32 a thread,
// as the single-simulation passes; the round kernel on labels holds 48).
#pragma once

#include "vd_batch_engine.cuh"
#include "vd_pass_pk.cuh"

namespace vdb {

// A thread's quads of one tile on words of layout M: rows ybase, ybase + 4,
// ... (n_rows of them).  MODE 0: the frame's first such pass (labels in,
// words out); 1 words to words; 2 the last (words in, labels out).  `in`: the
// tile and every neighbour at offset k lie inside the map (no range tests;
// tiles at the border take the out-of-line path).  One function per
// combination, out of line, so that each keeps a register allocation of its
// own inside the dispatching kernel.
template <int NB, int KS, int M, int MODE, bool DEDUP>
__device__ __noinline__ void pk_tile_rows(const vdk::PassArgs a, int x0, int ybase, int n_rows, bool in) {
  for (int i = 0; i < n_rows; ++i) {
    const int y = ybase + 4 * i;
    if (x0 >= a.pitch || y >= a.h) continue;
    if (!in) vdk::pk_edge_quad<NB, KS, M, MODE, DEDUP>(a, x0, y);
    else if (MODE == 0) vdk::pk_first_quad<NB, KS, M, DEDUP, true>(a, x0, y);
    else vdk::pk_quad<NB, KS, M, MODE == 1, true>(a, x0, y);
  }
}

template <int NB, int KS, int M>
__device__ __forceinline__ void pk_tile_nb(const vdk::PassArgs& a, int x0, int ybase, int n_rows, int mode,
                                           bool dedup, bool in) {
  if (mode == 0) {
    if (dedup) pk_tile_rows<NB, KS, M, 0, true>(a, x0, ybase, n_rows, in);
    else pk_tile_rows<NB, KS, M, 0, false>(a, x0, ybase, n_rows, in);
  } else if (mode == 1) {
    pk_tile_rows<NB, KS, M, 1, false>(a, x0, ybase, n_rows, in);
  } else {
    pk_tile_rows<NB, KS, M, 2, false>(a, x0, ybase, n_rows, in);
  }
}

// Round r's tiles [t0, t0 + gridDim.x), all of simulations whose pass r runs
// on words of layout M.
template <int M>
__global__ void __launch_bounds__(kThreads, 8) k_batch_round_pk(BatchArgs A, int r, int t0) {
  const TileAt at = tile_at(A, r, t0 + static_cast<int>(blockIdx.x));
  const SimDesc* sd = at.sd;
  const vdk::PassArgs a = round_args(sd, A.sched, r);
  const int k = a.k;
  const int nb = sd->nbs[A.sched][r];
  const int ksel = (k == 1) ? 1 : (k == 2 ? 2 : 0);
  const int rows = 4 * A.rows_per_thread;
  const int x0 = 4 * (at.tx * kQuadsX + static_cast<int>(threadIdx.x % kQuadsX));
  const int pkf = sd->pk_first[A.sched];
  const int mode = r == pkf ? 0 : (r == sd->n_pass[A.sched] - 1 ? 2 : 1);
  const bool dedup = sd->dedup[A.sched] != 0;
  const int xb = 4 * at.tx * kQuadsX, yb = at.ty * rows;
  const bool in = xb - k >= 0 && xb + 4 * kQuadsX + k <= a.w && yb - k >= 0 && yb + rows + k <= a.h;
  const int ybase = yb + static_cast<int>(threadIdx.x / kQuadsX);
  const int n_rows = A.rows_per_thread;
  switch (nb * 4 + ksel) {
    case 0: pk_tile_nb<vdk::kMoore, 0, M>(a, x0, ybase, n_rows, mode, dedup, in); break;
    case 1: pk_tile_nb<vdk::kMoore, 1, M>(a, x0, ybase, n_rows, mode, dedup, in); break;
    case 2: pk_tile_nb<vdk::kMoore, 2, M>(a, x0, ybase, n_rows, mode, dedup, in); break;
    case 4: pk_tile_nb<vdk::kVonNeumann, 0, M>(a, x0, ybase, n_rows, mode, dedup, in); break;
    case 5: pk_tile_nb<vdk::kVonNeumann, 1, M>(a, x0, ybase, n_rows, mode, dedup, in); break;
    default: pk_tile_nb<vdk::kVonNeumann, 2, M>(a, x0, ybase, n_rows, mode, dedup, in); break;
  }
}

template <int M>
int launch_round_pk_m(const BatchArgs& A, int r, int t0, int n_tiles, cudaStream_t st) {
  k_batch_round_pk<M><<<n_tiles, kThreads, 0, st>>>(A, r, t0);
  return vd_cuda_check(cudaGetLastError(), "batched packed round launch");
}

}  // namespace vdb
