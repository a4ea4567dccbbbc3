// vd_batch_engine.cuh -- device code and launch planning shared by the
// batched engine (vd_batch.cu) and the server (vd_serve.cu).
//
// Simulations are described by SimDesc records in device memory; a launch
// is planned on the host (HostPlan: active simulations, their 256-seed
// blocks, and per pass round the tiles of every simulation that still has a
// pass to run) and executed by the phase kernels below.  Every simulation
// runs exactly the per-thread code of the single-simulation passes
// (vdk::pass_quad) on its own maps, so its results do not depend on which
// other simulations share the launch.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace vdb {

constexpr int kMaxPasses = 20;   // 15 (side 32768) + 2 extra, with margin
constexpr int kThreads = 256;    // 64 quads x 4 rows per block
constexpr int kQuadsX = 64;

struct SimDesc {
  int w, h, pitch, n;
  int32_t* map[2];
  int2* seeds;
  int2* table;   // entry 0 = sentinel; the pass table is table + 1
  uint32_t* ptable;  // packed positions, entry 0 = far position; used as ptable + 1
  uint32_t cap, mul;       // clamped-key parameters (cap = 0: unusable)
  uint32_t clampmask[2];   // bit r: pass r of the schedule uses clamped keys
  uint32_t bytemask[2];    // bit r: pass r uses the byte-offset key (its fallback: the clamped one)
  int dedup[2];            // 1: the schedule's passes de-duplicate repeated table gathers
  int pk_first[2];         // passes [pk_first, n_pass) run on position-tagged words (n_pass: none)
  int pk_m;                // their word layout (8, 7 or 6; 0: none), dJFA schedule
  uint2* pkf;              // n + 1 seed entries of the wide layouts, [0] far; written by the stamp
  uint32_t bmul, bwin_bias, bwin_mask, blim;  // byte-offset key of the first such pass (PassArgs fields)
  int seed_off;
  int cur;
  long long step;      // moves drawn so far (the RNG step of the next move)
  int n_pass[2];       // [0] dJFA schedule, [1] JFA schedule
  int ks[2][kMaxPasses];
  int nbs[2][kMaxPasses];
};

struct Barrier {
  unsigned int count;
  unsigned int gen;
  int err;   // sticky: 1 = a bounded wait ran out
  int pad;
};

// One planned launch.  All arrays live in device memory.
struct BatchArgs {
  SimDesc* sims;
  const int* act;        // active simulations
  int n_act;
  const int2* sblk;      // (sim, first seed) per 256-seed block of the active simulations
  int n_sblk;
  const int* round_tiles;   // tiles per round
  const int* round_off;     // entries of round r: [round_off[r], round_off[r+1])
  const int2* entries;      // (sim, first tile of that sim in the round)
  int rounds;
  int sched;                // 0 = dJFA schedule, 1 = JFA schedule
  int mark;                 // 1: overwrite seed pixels before the minimum (dJFA); 0: JFA (map pre-filled)
  int move;                 // 1: move seeds first
  const int2* dxy;          // given moves (concatenated, seed_off indexed) or null for RNG
  int max_disp;
  unsigned long long rng_seed;
  int rows_per_thread;
  Barrier* bar;
  long long timeout_ns;
  int test_skip_arrive;
  int coh_byte;  // persistent launch: the byte-offset key on the passes that take it (else clamped)
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier with a bounded wait.  Returns false once any block's wait has
// run out (then every block returns at its next barrier).
static __device__ bool grid_sync(const BatchArgs& A, bool skip_arrive) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile int* err = &A.bar->err;
    int ok = (*err == 0);
    if (ok) {
      volatile unsigned int* gen = &A.bar->gen;
      const unsigned int g = *gen;
      __threadfence();
      bool released = false;
      if (!skip_arrive) {
        const unsigned int arrived = atomicAdd(&A.bar->count, 1u);
        if (arrived == gridDim.x - 1) {
          atomicExch(&A.bar->count, 0u);
          __threadfence();
          atomicAdd(&A.bar->gen, 1u);
          released = true;
        }
      }
      if (!released) {
        const unsigned long long t0 = global_ns();
        while (*gen == g && *err == 0) {
          if (global_ns() - t0 > static_cast<unsigned long long>(A.timeout_ns)) {
            atomicCAS(&A.bar->err, 0, 1);
            break;
          }
          __nanosleep(200);
        }
      }
      __threadfence();
      ok = (*err == 0);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---- phases ---------------------------------------------------------------

__device__ __forceinline__ void move_mark_block(const BatchArgs& A, int sb) {
  const int2 blk = A.sblk[sb];
  SimDesc* sd = A.sims + blk.x;
  const int k = blk.y + static_cast<int>(threadIdx.x);
  if (k >= sd->n) return;
  int2 p = sd->seeds[k];
  if (A.move) {
    long long dx, dy;
    if (A.dxy != nullptr) {
      const int2 d = A.dxy[sd->seed_off + k];
      dx = d.x;
      dy = d.y;
    } else {
      const uint64_t key = vdk::splitmix64(A.rng_seed, static_cast<uint64_t>(blk.x));
      const uint64_t step = static_cast<uint64_t>(sd->step);
      dx = vdk::rng_disp(key, step, static_cast<uint64_t>(k), 0, A.max_disp);
      dy = vdk::rng_disp(key, step, static_cast<uint64_t>(k), 1, A.max_disp);
    }
    long long x = p.x + dx, y = p.y + dy;
    x = x < 0 ? 0 : (x > sd->w - 1 ? sd->w - 1 : x);
    y = y < 0 ? 0 : (y > sd->h - 1 ? sd->h - 1 : y);
    p.x = static_cast<int>(x);
    p.y = static_cast<int>(y);
    sd->seeds[k] = p;
    sd->table[k + 1] = vdk::table_entry(p);
    sd->ptable[k + 1] = vdk::pack_pos(p.x, p.y);
  }
  if (A.mark) sd->map[sd->cur][static_cast<int64_t>(p.y) * sd->pitch + p.x] = k;
}

__device__ __forceinline__ void stamp_min_block(const BatchArgs& A, int sb) {
  const int2 blk = A.sblk[sb];
  const SimDesc* sd = A.sims + blk.x;
  const int k = blk.y + static_cast<int>(threadIdx.x);
  if (k >= sd->n) return;
  const int2 p = sd->seeds[k];
  atomicMin(reinterpret_cast<unsigned int*>(sd->map[sd->cur] + static_cast<int64_t>(p.y) * sd->pitch + p.x),
            static_cast<unsigned int>(k));
  // the seed entries of a wide word layout (as k_stamp_min: bit 24 set, x and
  // y modulo 2^m at [24 - m, 24) and [32 - m, 32)), for this step's passes
  const int m = A.sched == 0 ? sd->pk_m : 0;
  if (m == 6 || m == 7) {
    const uint32_t xm = (1u << m) - 1u;
    const uint32_t f = (1u << 24) | ((static_cast<uint32_t>(p.x) & xm) << (24 - m)) |
                       ((static_cast<uint32_t>(p.y) & xm) << (32 - m));
    sd->pkf[k + 1] = make_uint2(vdk::pack_pos(p.x, p.y), f);
    if (k == 0) sd->pkf[0] = make_uint2(sd->ptable[0], 0u);
  }
}

// One quad of a pass in a 32-bit key form, dispatched on the neighbourhood and step.
template <int METRIC, bool COH, bool DEDUP, bool MCAP>
__device__ __forceinline__ void tile_quad32(const vdk::PassArgs& a, int x0, int y, int nb, int ksel) {
  switch (nb * 4 + ksel) {
    case 0: vdk::pass_quad_clamped<vdk::kMoore, 0, COH, METRIC, DEDUP, MCAP>(a, x0, y); break;
    case 1: vdk::pass_quad_clamped<vdk::kMoore, 1, COH, METRIC, DEDUP, MCAP>(a, x0, y); break;
    case 2: vdk::pass_quad_clamped<vdk::kMoore, 2, COH, METRIC, DEDUP, MCAP>(a, x0, y); break;
    case 4: vdk::pass_quad_clamped<vdk::kVonNeumann, 0, COH, METRIC, DEDUP, MCAP>(a, x0, y); break;
    case 5: vdk::pass_quad_clamped<vdk::kVonNeumann, 1, COH, METRIC, DEDUP, MCAP>(a, x0, y); break;
    default: vdk::pass_quad_clamped<vdk::kVonNeumann, 2, COH, METRIC, DEDUP, MCAP>(a, x0, y); break;
  }
}

// One quad of a pass, dispatched on the key form, neighbourhood and step
// (mcap: the clamped Manhattan form, for more than 2^15 labels).
template <int METRIC, bool COH, bool DEDUP>
__device__ __forceinline__ void tile_quad(const vdk::PassArgs& a, int x0, int y, bool clamp, bool mcap, int nb,
                                          int ksel) {
  if (clamp) {
    if (METRIC == vdk::kManhattan && mcap) tile_quad32<METRIC, COH, DEDUP, true>(a, x0, y, nb, ksel);
    else tile_quad32<METRIC, COH, DEDUP, false>(a, x0, y, nb, ksel);
    return;
  }
  switch (nb * 4 + ksel) {
    case 0: vdk::pass_quad<vdk::kMoore, METRIC, 0, COH, DEDUP>(a, x0, y); break;
    case 1: vdk::pass_quad<vdk::kMoore, METRIC, 1, COH, DEDUP>(a, x0, y); break;
    case 2: vdk::pass_quad<vdk::kMoore, METRIC, 2, COH, DEDUP>(a, x0, y); break;
    case 4: vdk::pass_quad<vdk::kVonNeumann, METRIC, 0, COH, DEDUP>(a, x0, y); break;
    case 5: vdk::pass_quad<vdk::kVonNeumann, METRIC, 1, COH, DEDUP>(a, x0, y); break;
    default: vdk::pass_quad<vdk::kVonNeumann, METRIC, 2, COH, DEDUP>(a, x0, y); break;
  }
}

// One quad of a pass in the byte-offset key form (Euclidean, below 2^16 seeds).
template <bool COH, bool DEDUP>
__device__ __forceinline__ void tile_quad8(const vdk::PassArgs& a, int x0, int y, int nb, int ksel) {
  switch (nb * 4 + ksel) {
    case 0: vdk::pass_quad_byte<vdk::kMoore, 0, COH, DEDUP>(a, x0, y); break;
    case 1: vdk::pass_quad_byte<vdk::kMoore, 1, COH, DEDUP>(a, x0, y); break;
    case 2: vdk::pass_quad_byte<vdk::kMoore, 2, COH, DEDUP>(a, x0, y); break;
    case 4: vdk::pass_quad_byte<vdk::kVonNeumann, 0, COH, DEDUP>(a, x0, y); break;
    case 5: vdk::pass_quad_byte<vdk::kVonNeumann, 1, COH, DEDUP>(a, x0, y); break;
    default: vdk::pass_quad_byte<vdk::kVonNeumann, 2, COH, DEDUP>(a, x0, y); break;
  }
}

// Round r's tile t: its simulation and tile coordinates (the entry holding
// tile t is the last one whose first tile is <= t).
struct TileAt {
  const SimDesc* sd;
  int tx, ty;
};

__device__ __forceinline__ TileAt tile_at(const BatchArgs& A, int r, int t) {
  int lo = A.round_off[r], hi = A.round_off[r + 1] - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.entries[mid].y <= t) lo = mid;
    else hi = mid - 1;
  }
  const int2 e = A.entries[lo];
  TileAt at;
  at.sd = A.sims + e.x;
  const int lt = t - e.y;
  const int tiles_x = (at.sd->pitch + 4 * kQuadsX - 1) / (4 * kQuadsX);
  at.tx = lt % tiles_x;
  at.ty = lt / tiles_x;
  return at;
}

// The single-simulation pass arguments of simulation sd's pass r.
__device__ __forceinline__ vdk::PassArgs round_args(const SimDesc* sd, int sched, int r) {
  vdk::PassArgs a;
  a.src = sd->map[(sd->cur + r) & 1];
  a.dst = sd->map[(sd->cur + r + 1) & 1];
  a.table = sd->table + 1;
  a.ptable = sd->ptable + 1;
  a.cap = sd->cap;
  a.mul = sd->mul;
  a.bmul = sd->bmul;
  a.bwin_bias = sd->bwin_bias;
  a.bwin_mask = sd->bwin_mask;
  a.blim = sd->blim;
  a.pkf = sd->pkf;
  a.n_seeds = static_cast<uint32_t>(sd->n);
  a.w = sd->w;
  a.h = sd->h;
  a.y0 = 0;
  a.y_end = sd->h;
  a.pitch = sd->pitch;
  a.k = sd->ks[sched][r];
  a.band_m = 1;
  a.band_t = 1;
  return a;
}

// A tile of a pass on labels.  (Tiles of passes on position-tagged words run
// in k_batch_round_pk, vd_batch_pk.cuh.)
template <int METRIC, bool COH>
__device__ __forceinline__ void round_tile(const BatchArgs& A, int r, int t) {
  const TileAt at = tile_at(A, r, t);
  const SimDesc* sd = at.sd;
  const vdk::PassArgs a = round_args(sd, A.sched, r);
  const int k = a.k;
  const int nb = sd->nbs[A.sched][r];
  const int x0 = 4 * (at.tx * kQuadsX + static_cast<int>(threadIdx.x % kQuadsX));
  const int ksel = (k == 1) ? 1 : (k == 2 ? 2 : 0);
  const bool clamp = (sd->clampmask[A.sched] >> r) & 1u;
  const int rows = 4 * A.rows_per_thread;
  const bool dedup = sd->dedup[A.sched] != 0;
  const bool mcap = sd->mul > (1u << 15);
  const bool byte = (COH ? A.coh_byte : true) && METRIC == vdk::kEuclid && ((sd->bytemask[A.sched] >> r) & 1u);
  for (int i = 0; i < A.rows_per_thread; ++i) {
    const int y = at.ty * rows + static_cast<int>(threadIdx.x / kQuadsX) + 4 * i;
    if (x0 >= a.pitch || y >= a.h) continue;
    if (byte) {
      if (dedup) tile_quad8<COH, true>(a, x0, y, nb, ksel);
      else tile_quad8<COH, false>(a, x0, y, nb, ksel);
    } else if (dedup) {
      tile_quad<METRIC, COH, true>(a, x0, y, clamp, mcap, nb, ksel);
    } else {
      tile_quad<METRIC, COH, false>(a, x0, y, clamp, mcap, nb, ksel);
    }
  }
}

__device__ __forceinline__ void finish_sim(const BatchArgs& A, int i) {
  SimDesc* sd = A.sims + A.act[i];
  sd->cur ^= (sd->n_pass[A.sched] & 1);
  if (A.move) sd->step += 1;
}

// ---- launch-per-phase kernels --------------------------------------------

static __global__ void __launch_bounds__(kThreads) k_batch_move_mark(BatchArgs A) {
  move_mark_block(A, blockIdx.x);
}

static __global__ void __launch_bounds__(kThreads) k_batch_min(BatchArgs A) { stamp_min_block(A, blockIdx.x); }

// Round r's tiles from t0 on (the ones on labels).
template <int METRIC>
__global__ void __launch_bounds__(kThreads, 5) k_batch_round(BatchArgs A, int r, int t0) {
  round_tile<METRIC, false>(A, r, t0 + static_cast<int>(blockIdx.x));
}

// Round r's tiles [t0, t0 + n_tiles), all of simulations whose pass r runs on
// position-tagged words of layout m (8, 7, 6): vd_batch_pk<m>.cu.
int launch_round_pk(int m, const BatchArgs& A, int r, int t0, int n_tiles, cudaStream_t st);

static __global__ void k_batch_finish(BatchArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < A.n_act) finish_sim(A, i);
}

// ---- the persistent kernel -------------------------------------------------

// MINB: resident blocks per SM the register budget is cut for (4: 64
// registers a thread; 5: 48, as the per-round kernel).
template <int METRIC, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_batch_persistent(BatchArgs A) {
  if (*reinterpret_cast<volatile int*>(&A.bar->err) != 0) return;
  if (A.move || A.mark) {
    for (int sb = blockIdx.x; sb < A.n_sblk; sb += gridDim.x) move_mark_block(A, sb);
    if (!grid_sync(A, A.test_skip_arrive && blockIdx.x == 0)) return;
  }
  for (int sb = blockIdx.x; sb < A.n_sblk; sb += gridDim.x) stamp_min_block(A, sb);
  if (!grid_sync(A, false)) return;
  for (int r = 0; r < A.rounds; ++r) {
    const int nt = A.round_tiles[r];
    // maps are rewritten between barriers of this launch: coherent loads
    for (int t = blockIdx.x; t < nt; t += gridDim.x) round_tile<METRIC, true>(A, r, t);
    if (!grid_sync(A, false)) return;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n_act; i += gridDim.x * blockDim.x) finish_sim(A, i);
}

}  // namespace vdb

namespace vdb {

struct HostPlan {
  std::vector<int> act;
  std::vector<int2> sblk;
  std::vector<int> round_tiles, round_off;
  // per word layout (8, 7, 6) and round: the round's first tiles, of
  // simulations whose pass r runs on words of that layout, in that order
  std::vector<int> pk_tiles[3];
  std::vector<int2> entries;
  int rounds = 0;
  int64_t pixel_passes = 0;
};

inline int tiles_of(const SimDesc& s, int rpt) {
  const int tx = (s.pitch + 4 * kQuadsX - 1) / (4 * kQuadsX);
  const int ty = (s.h + 4 * rpt - 1) / (4 * rpt);
  return tx * ty;
}

inline HostPlan make_plan(const std::vector<SimDesc>& sims, const std::vector<int>& act, int sched, int rpt) {
  HostPlan p;
  p.act = act;
  for (int i : act) {
    const SimDesc& s = sims[i];
    for (int first = 0; first < s.n; first += kThreads) p.sblk.push_back(make_int2(i, first));
    p.rounds = std::max(p.rounds, s.n_pass[sched]);
    p.pixel_passes += static_cast<int64_t>(s.w) * s.h * s.n_pass[sched];
  }
  p.round_off.push_back(0);
  for (int r = 0; r < p.rounds; ++r) {
    int t = 0;
    // simulations whose pass r runs on words of layout 8, 7, 6, then the rest
    for (int g = 0; g < 4; ++g) {
      const int t_g = t;
      for (int i : act) {
        const SimDesc& s = sims[i];
        if (s.n_pass[sched] <= r) continue;
        const bool words = s.pk_first[sched] <= r;
        if (g < 3 ? (words && s.pk_m == 8 - g) : !words) {
          p.entries.push_back(make_int2(i, t));
          t += tiles_of(s, rpt);
        }
      }
      if (g < 3) p.pk_tiles[g].push_back(t - t_g);
    }
    p.round_tiles.push_back(t);
    p.round_off.push_back(static_cast<int>(p.entries.size()));
  }
  return p;
}


// Clamped-key parameters and per-pass choices of one simulation for one
// schedule (sched 0 = dJFA, 1 = JFA) under `metric`.
// Per-schedule key form (clamped 32-bit or exact, per pass) and gather
// de-duplication (the single-simulation auto rules).
inline void set_clamp(SimDesc& s, int sched, int32_t metric, int clamp_option, int packed_option = -1) {
  const int lb = vdi::label_bits(s.n);
  s.mul = lb >= 32 ? 0u : (1u << lb);
  s.cap = lb >= 4 ? static_cast<uint32_t>((uint64_t{1} << (32 - lb)) - 1) : 0u;
  uint32_t mask = 0;
  for (int r = 0; r < s.n_pass[sched] && r < 32; ++r)
    if (vdi::use_clamp(clamp_option, metric, s.n, s.ks[sched][r], sched == 0)) mask |= 1u << r;
  s.clampmask[sched] = mask;
  s.dedup[sched] = vdi::use_dedup(-1, s.w, s.h, s.n, sched == 0) ? 1 : 0;
  // Byte-offset keys (launch-per-round mode) on the clamped dJFA passes below
  // 2^16 seeds whose mean cell radius is at most 40 pixels, at steps
  // 2 .. 128.  Unlike a lone simulation no map-size bound: a round launch
  // holds every simulation's tiles.  Not k = 1: at the round kernel's 48
  // registers the byte form is no faster there (it is at the 32 registers of
  // a lone simulation's pass).  256 simulations: 9.12 -> 8.80 ms a step.
  uint32_t bmask = 0;
  const bool small_cells = static_cast<double>(s.w) * s.h <= 3.141592653589793 * 40.0 * 40.0 * s.n;
  if (sched == 0 && metric == VD_METRIC_EUCLID && s.n < 65536 && lb >= 4 && small_cells) {
    for (int r = 0; r < s.n_pass[sched] && r < 32; ++r) {
      const int k = s.ks[sched][r];
      if (((mask >> r) & 1u) && k > 1 && k <= 128) bmask |= 1u << r;
    }
  }
  s.bytemask[sched] = bmask;
  // Position-tagged words (launch-per-round mode): the dJFA frame's last
  // passes with k = 1, 2 or a multiple of 4, at least two of them, at steps
  // up to 128 and twice the layout's and the first pass's byte-key windows,
  // under the byte-offset key's mean-radius bound taken at the layout's
  // window, up to 2^18 seeds (word layouts 8, 7, 6 as a single simulation's;
  // the wide ones read the 8-byte seed entries the stamp writes).  The
  // frame's first such pass folds with the byte-offset key: its window and
  // label field (narrow below 2^16 seeds) go to the descriptor.
  // packed_option: -1 auto, 0 never.
  int pkf = s.n_pass[sched];
  int blb = 16;
  const int hb = vdi::byte_key_window(s.n, &blb);
  s.bmul = blb >= 32 ? 0u : (1u << blb);
  s.bwin_bias = static_cast<uint32_t>(hb) * 0x10001u;
  s.bwin_mask = hb ? (0xFFFFu & ~(2u * hb - 1u)) * 0x10001u : 0xFFFFFFFFu;
  s.blim = static_cast<uint32_t>(hb) * static_cast<uint32_t>(hb) * s.bmul;
  if (sched == 0) {
    s.pk_m = 0;
    const int lay = vdi::pk_bits(s.n);
    const int hp = lay ? 1 << (lay - 1) : 0;
    const double r_max = 40.0 * hp / 128.0;
    if (packed_option != 0 && metric == VD_METRIC_EUCLID && lay >= 6 && lb >= 4 && hb >= 32 &&
        static_cast<double>(s.w) * s.h <= 3.141592653589793 * r_max * r_max * s.n) {
      auto ok = [&](int k) { return (k == 1 || k == 2 || k % 4 == 0) && k <= 128 && k <= 2 * hp && k <= 2 * hb; };
      while (pkf > 0 && ok(s.ks[sched][pkf - 1])) --pkf;
      if (s.n_pass[sched] - pkf < 2) pkf = s.n_pass[sched];
      if (pkf < s.n_pass[sched]) s.pk_m = lay;
    }
  }
  s.pk_first[sched] = pkf;
}

// A pinned host staging buffer and a device buffer for one plan.
struct PlanSlot {
  int* d = nullptr;
  int* h = nullptr;
  size_t cap = 0;  // ints
  void release() {
    cudaFree(d);
    cudaFreeHost(h);
    d = nullptr;
    h = nullptr;
    cap = 0;
  }
};

// Packs a plan into `slot` and queues its upload on `st`; fills the plan
// fields of *A.  The caller guarantees that no launch still reads the slot
// (and that the host staging buffer's previous upload has run).
inline int plan_upload(PlanSlot& slot, const HostPlan& p, SimDesc* d_sims, cudaStream_t st, BatchArgs* A) {
  const size_t need = p.act.size() + 2 * p.sblk.size() + p.round_tiles.size() + p.round_off.size() +
                      2 * p.entries.size() + 8;
  if (need > slot.cap) {
    slot.release();
    const size_t cap = std::max(need, static_cast<size_t>(1024));
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&slot.d), sizeof(int) * cap);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&slot.h), sizeof(int) * cap);
    if (e != cudaSuccess) {
      slot.release();
      return vd_cuda_check(e, "plan buffers");
    }
    slot.cap = cap;
  }
  int* h = slot.h;
  size_t o = 0;
  auto put = [&](const int* src, size_t n) {
    std::memcpy(h + o, src, sizeof(int) * n);
    o += n;
  };
  // int2 sections are read with 8-byte loads: start them on an even int
  auto align2 = [&]() { o = (o + 1) & ~static_cast<size_t>(1); };
  const size_t o_act = o;
  put(p.act.data(), p.act.size());
  align2();
  const size_t o_sblk = o;
  put(reinterpret_cast<const int*>(p.sblk.data()), 2 * p.sblk.size());
  const size_t o_rt = o;
  put(p.round_tiles.data(), p.round_tiles.size());
  const size_t o_ro = o;
  put(p.round_off.data(), p.round_off.size());
  align2();
  const size_t o_ent = o;
  put(reinterpret_cast<const int*>(p.entries.data()), 2 * p.entries.size());
  if ((o_sblk | o_ent) & 1) return vd_fail(VD_ECUDA, "internal: misaligned plan section");
  const int rc = vd_cuda_check(cudaMemcpyAsync(slot.d, h, sizeof(int) * o, cudaMemcpyHostToDevice, st), "upload plan");
  if (rc) return rc;
  A->sims = d_sims;
  A->act = slot.d + o_act;
  A->n_act = static_cast<int>(p.act.size());
  A->sblk = reinterpret_cast<const int2*>(slot.d + o_sblk);
  A->n_sblk = static_cast<int>(p.sblk.size());
  A->round_tiles = slot.d + o_rt;
  A->round_off = slot.d + o_ro;
  A->entries = reinterpret_cast<const int2*>(slot.d + o_ent);
  A->rounds = p.rounds;
  return VD_OK;
}

// One launch per phase and pass round (stream-ordered).
inline int launch_rounds(const HostPlan& p, const BatchArgs& A, int metric, cudaStream_t st, int64_t* launches) {
  if (A.n_sblk > 0 && (A.move || A.mark)) {
    k_batch_move_mark<<<A.n_sblk, kThreads, 0, st>>>(A);
    ++*launches;
  }
  if (A.n_sblk > 0) {
    k_batch_min<<<A.n_sblk, kThreads, 0, st>>>(A);
    ++*launches;
  }
  for (int r = 0; r < p.rounds; ++r) {
    int t0 = 0;
    for (int g = 0; g < 3; ++g) {
      const int n = p.pk_tiles[g][r];
      if (n <= 0) continue;
      const int rc = launch_round_pk(8 - g, A, r, t0, n, st);
      if (rc) return rc;
      ++*launches;
      t0 += n;
    }
    const int rest = p.round_tiles[r] - t0;
    if (rest <= 0) continue;
    if (metric == VD_METRIC_MANHATTAN)
      k_batch_round<vdk::kManhattan><<<rest, kThreads, 0, st>>>(A, r, t0);
    else
      k_batch_round<vdk::kEuclid><<<rest, kThreads, 0, st>>>(A, r, t0);
    ++*launches;
  }
  if (A.n_act > 0) {
    k_batch_finish<<<(A.n_act + 255) / 256, 256, 0, st>>>(A);
    ++*launches;
  }
  return vd_cuda_check(cudaGetLastError(), "batch launch");
}

inline BatchArgs make_args(int rows_per_thread, Barrier* bar, long long timeout_ns, int test_skip_arrive,
                           int coh_byte) {
  BatchArgs A;
  std::memset(&A, 0, sizeof(A));
  A.coh_byte = coh_byte;
  A.rows_per_thread = rows_per_thread;
  A.bar = bar;
  A.timeout_ns = timeout_ns;
  A.test_skip_arrive = test_skip_arrive;
  return A;
}

}  // namespace vdb
