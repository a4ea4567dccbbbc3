// vd_api.cu -- the C ABI of include/vd.h for one simulation: context state,
// schedules (Eq. 2, Eq. 3-4), launch planning of the jump passes, copies and
// error reporting.  All pixel work runs in the kernels of vd_kernels.cuh.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace {

thread_local std::string g_error;

}  // namespace

int vd_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

int vd_cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return VD_OK;
  return vd_fail(e == cudaErrorMemoryAllocation ? VD_ENOMEM : VD_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

extern "C" const char* vd_last_error(void) { return g_error.c_str(); }

extern "C" int vd_abi_version(void) { return 1; }

// ---------------------------------------------------------------------------
// Schedules
// ---------------------------------------------------------------------------

namespace vdi {

int ceil_log2(int64_t v) {
  int e = 0;
  while ((int64_t{1} << e) < v) ++e;
  return e;
}

// Eq. 2: k_1 = 2^(ceil(log2 N) - 1), N = max(w, h); 0 when N = 1 (no pass).
int32_t jfa_first_step(int32_t w, int32_t h) {
  const int e = ceil_log2(w > h ? w : h);
  return e == 0 ? 0 : (int32_t{1} << (e - 1));
}

// Eq. 3-4 in exact integers: the least power of two P with P^2 s >= 4 w h
// (P >= 2 L_avg) and P >= d_max, capped at k_1.  Dense seeds can make the
// exponent negative (no pass).
int32_t djfa_first_step(int32_t w, int32_t h, int64_t s, int32_t d_max) {
  const int32_t k1 = jfa_first_step(w, h);
  if (s <= 0) return k1;
  const int64_t area4 = 4 * static_cast<int64_t>(w) * h;
  int e;
  if (s >= area4) {
    // P <= 1: find the least e <= 0 with s * 4^e >= area4, i.e. s >= area4 * 4^-e.
    e = 0;
    while (e > -31 && (s >> (2 * (1 - e))) >= area4) --e;
  } else {
    e = 0;
    while ((s << (2 * e)) < area4) ++e;
  }
  if (d_max > 0) {
    const int ed = ceil_log2(d_max);
    if (ed > e) e = ed;
  }
  if (e < 0) return 0;
  const int64_t p = int64_t{1} << e;
  return static_cast<int32_t>(p > k1 ? k1 : p);
}

int fill_schedule(int32_t first, int32_t vn_waves, int32_t extra, int32_t* ks, int32_t* nbs,
                  int32_t cap) {
  int n = 0;
  for (int32_t k = first; k >= 1; k >>= 1, ++n) {
    if (n < cap) {
      ks[n] = k;
      nbs[n] = n < vn_waves ? VD_NB_VON_NEUMANN : VD_NB_MOORE;
    }
  }
  for (int32_t e = extra; e >= 1; --e, ++n) {
    if (n < cap) {
      ks[n] = int32_t{1} << (e - 1);
      nbs[n] = VD_NB_MOORE;
    }
  }
  return n;
}

}  // namespace vdi

static bool bad_side(int32_t v) { return v < 1 || v > VD_MAX_SIDE; }

extern "C" int vd_jfa_schedule(int32_t w, int32_t h, int32_t extra, int32_t* ks, int32_t* nbs,
                               int32_t cap) {
  if (bad_side(w) || bad_side(h)) return vd_fail(VD_EINVAL, "grid %dx%d outside [1, %d]", w, h, VD_MAX_SIDE);
  if (extra < 0 || extra > 2) return vd_fail(VD_EINVAL, "extra_passes %d outside [0, 2]", extra);
  if (cap < 0 || (cap > 0 && (!ks || !nbs))) return vd_fail(VD_EINVAL, "bad output arrays");
  return vdi::fill_schedule(vdi::jfa_first_step(w, h), 0, extra, ks, nbs, cap);
}

extern "C" int vd_djfa_schedule(int32_t w, int32_t h, int64_t s, int32_t d_max, int32_t vn_waves,
                                int32_t extra, int32_t* ks, int32_t* nbs, int32_t cap) {
  if (bad_side(w) || bad_side(h)) return vd_fail(VD_EINVAL, "grid %dx%d outside [1, %d]", w, h, VD_MAX_SIDE);
  if (s < 1) return vd_fail(VD_EINVAL, "n_seeds %lld < 1", static_cast<long long>(s));
  if (d_max < 0 || vn_waves < 0) return vd_fail(VD_EINVAL, "d_max/vn_waves must be >= 0");
  if (extra < 0 || extra > 2) return vd_fail(VD_EINVAL, "extra_passes %d outside [0, 2]", extra);
  if (cap < 0 || (cap > 0 && (!ks || !nbs))) return vd_fail(VD_EINVAL, "bad output arrays");
  return vdi::fill_schedule(vdi::djfa_first_step(w, h, s, d_max), vn_waves, extra, ks, nbs, cap);
}

// ---------------------------------------------------------------------------
// Launch planning shared with the batched engine
// ---------------------------------------------------------------------------

namespace vdi {

int ensure_smem(const void* fn, size_t bytes, size_t* done) {
  if (bytes <= 48 * 1024 || bytes <= *done) return VD_OK;
  const cudaError_t e =
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
  if (e != cudaSuccess) return vd_cuda_check(e, "cudaFuncSetAttribute(smem)");
  *done = bytes;
  return VD_OK;
}

// Launches `kern` on `st`.  With `pdl` the launch carries programmatic stream
// serialization: it may be scheduled while the previous kernel on the stream
// drains, and the kernel itself waits for that kernel (vdk::pdl_wait) before
// touching global memory.  Only kernels that begin with pdl_wait are launched
// this way.
template <typename... KArgs, typename... Args>
static cudaError_t launch_k(void (*kern)(KArgs...), dim3 g, dim3 b, cudaStream_t st, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

template <int NB, int METRIC, int KEY>
static cudaError_t launch_pass_t(int ksel, bool dedup, dim3 g, dim3 b, cudaStream_t st, bool pdl,
                                 const vdk::PassArgs& a) {
  if (dedup) {
    switch (ksel) {
      case 0: return launch_k(vdk::k_pass<NB, METRIC, 0, KEY, true>, g, b, st, pdl, a);
      case 1: return launch_k(vdk::k_pass<NB, METRIC, 1, KEY, true>, g, b, st, pdl, a);
      case 2: return launch_k(vdk::k_pass<NB, METRIC, 2, KEY, true>, g, b, st, pdl, a);
      default: break;  // any other step: scalar loads, never de-duplicated
    }
  }
  switch (ksel) {
    case 0: return launch_k(vdk::k_pass<NB, METRIC, 0, KEY>, g, b, st, pdl, a);
    case 1: return launch_k(vdk::k_pass<NB, METRIC, 1, KEY>, g, b, st, pdl, a);
    case 2: return launch_k(vdk::k_pass<NB, METRIC, 2, KEY>, g, b, st, pdl, a);
    default: return launch_k(vdk::k_pass<NB, METRIC, 3, KEY>, g, b, st, pdl, a);
  }
}

int label_bits(int32_t n) {
  int lb = 0;
  while ((int64_t{1} << lb) < n) ++lb;
  return lb;
}

bool use_clamp(int clamp_option, int32_t metric, int32_t n, int32_t k, bool djfa_frame) {
  (void)k;
  if (clamp_option == 0) return false;
  const int lb = label_bits(n);
  if (metric == VD_METRIC_MANHATTAN && lb <= 15) {
    // exact without a cap while d * 2^lb + label fits: every pass may use it
    return true;
  }
  if (lb < 4) return false;
  if (clamp_option == 1) return true;
  // Clamped keys (Euclidean; Manhattan beyond 2^15 labels), auto: dJFA
  // passes only.  The previous map is nearly right there, so quads almost
  // never reach the cap; in a JFA frame the early passes still see many empty
  // pixels, whose quads would be recomputed with the exact form.
  return djfa_frame;
}

// Byte-offset key: below 2^16 seeds a 16-bit label field and the window
// h = 128; from 2^16 seeds on (the wide form) lb bits with 2^lb > n (so that
// the all-ones field of an empty label names no seed) and the largest power
// of two h with (2h^2 + 1) * 2^lb <= 2^32, so that no key inside the window
// wraps.  Returns h, or 0 where the form does not apply.
int byte_key_window(int64_t n, int* lb_out) {
  if (n < 1) return 0;
  if (n < 65536) {
    if (lb_out) *lb_out = 16;
    return static_cast<int>(vdk::kByteWindow);
  }
  int lb = 0;
  while ((int64_t{1} << lb) <= n) ++lb;
  if (lb_out) *lb_out = lb;
  for (uint64_t h = 64; h >= 2; h >>= 1) {
    if (((2 * h * h + 1) << lb) <= (uint64_t{1} << 32)) return static_cast<int>(h);
  }
  return 0;
}

bool use_byte_key(int byte_option, int32_t metric, int32_t w, int32_t h, int32_t n, int32_t k,
                  bool djfa_frame) {
  // the form falls back to the clamped one, usable from 9 seeds on
  if (byte_option == 0 || metric != VD_METRIC_EUCLID || label_bits(n) < 4) return false;
  const int hw = byte_key_window(n, nullptr);
  if (hw == 0) return false;
  if (byte_option == 1) return true;
  if (!djfa_frame) return false;
  // auto: dJFA passes on maps of at least 2^21 pixels (on smaller ones a pass
  // is a wave or two of quads, and the winner check's second lookup adds more
  // latency than the saved instructions gain: 1024^2 2% slower, 2048^2 6%
  // faster on the GB300) with a mean cell radius of at most 40 pixels per 128
  // of window, so that nearly every pixel's winner lies inside the window and
  // recomputed quads stay rare (8192^2: 2^14 seeds, radius 36, 14% faster
  // with every pass on the byte-offset key; 2^10 seeds, radius 144, 1.7x
  // slower), at steps up to min(128, 2h): a seed k >= 256 away wraps to a
  // small byte offset, and such garbage keys would often beat the true
  // winner (the repair frame's JFA schedule, 2048^2: 0.275 -> 0.338 ms a step).
  // Not with windows narrower than 32 (2^20 seeds and more): moves of a few
  // pixels then already put the previous frame's seeds outside the window,
  // where their keys wrap (8192^2, 2^22 seeds, moves up to 16: 1.6x slower)
  if (static_cast<int64_t>(w) * h < (int64_t{1} << 21) || k > 128 || k > 2 * hw || hw < 32) return false;
  const double r_max = 40.0 * hw / 128.0;
  return static_cast<double>(w) * h <= 3.141592653589793 * r_max * r_max * n;
}

int launch_pass(const MapView& m, const int32_t* src, int32_t* dst, int32_t k, int32_t nb,
                int32_t metric, int64_t band_min_k, bool clamp, cudaStream_t st, bool pdl, bool dedup,
                bool byte_key, int blocked, int key_pack, int blk_min_blocks, bool sparse, int32_t y0,
                int32_t y1, int pass_bx, int tile_max_k, int tile_rows, int pk_m, int pk_mode) {
  if (y1 < 0) y1 = m.h;
  const bool rows_only = y0 != 0 || y1 != m.h;
  vdk::PassArgs a;
  a.src = src;
  a.dst = dst;
  a.table = m.table;
  a.ptable = m.ptable;
  a.pkf = m.pkf;
  {
    const int lb = label_bits(m.n);
    a.mul = lb >= 32 ? 0u : (1u << lb);
    a.cap = lb >= 4 ? static_cast<uint32_t>((uint64_t{1} << (32 - lb)) - 1) : 0u;
    int blb = 16;
    const uint32_t hw = static_cast<uint32_t>(byte_key_window(m.n, &blb));
    a.bmul = blb >= 32 ? 0u : (1u << blb);
    a.bwin_bias = hw * 0x10001u;
    a.bwin_mask = hw ? (0xFFFFu & ~(2u * hw - 1u)) * 0x10001u : 0xFFFFFFFFu;
    a.blim = hw * hw * a.bmul;
  }
  a.n_seeds = static_cast<uint32_t>(m.n);
  a.w = m.w;
  a.h = m.h;
  a.pitch = m.pitch;
  a.k = k;
  a.band_m = 1;
  a.band_t = 1;
  a.y0 = y0;
  a.y_end = y1;
  const int quads = m.pitch / 4;
  const int tile = (pass_bx == 32 || pass_bx == 128) ? pass_bx : 64;
  const int bx = quads < tile ? quads : tile;
  const int by = (pk_m ? pk_threads(nb, pk_mode) : vdk::kPassThreads) / bx;
  const int nrb = (y1 - y0 + by - 1) / by;
  dim3 block(bx, by);
  dim3 grid((quads + bx - 1) / bx, nrb);
  bool band = false;
  if (band_min_k < 0) {
    // auto: once the rows y-k .. y+k span more than a quarter of L2
    band = 2.0 * k * m.pitch * 4.0 >= 32.0 * 1024 * 1024;
  } else if (band_min_k > 0) {
    band = k >= band_min_k;
  }
  if (band && k % by == 0 && k / by > 1) {
    a.band_m = k / by;
    a.band_t = (nrb + a.band_m - 1) / a.band_m;
    grid.y = a.band_m * a.band_t;
  }
  const int ksel = (k % 4 == 0) ? 0 : (k == 1 ? 1 : (k == 2 ? 2 : 3));
  // key form: 0 exact 64-bit, 1 32-bit, 2 clamped Manhattan 32-bit, 3 byte-offset
  int key = 0;
  if (clamp) {
    if (metric == VD_METRIC_MANHATTAN) key = label_bits(m.n) <= 15 ? 1 : 2;
    else if (a.cap != 0) key = 1;
  }
  if (byte_key && metric == VD_METRIC_EUCLID && a.cap != 0 && a.bwin_bias != 0) key = m.n < 65536 ? 3 : 4;
  // the position-tagged passes of a dJFA frame (chosen by run_passes)
  if (pk_m) {
    // the first pass folds with a byte-offset key (the narrow one for the
    // 8-bit layout; either for the wide ones; the split layout's with the
    // clamped key)
    const bool first_ok = pk_m == 4 ? a.cap != 0 : key >= 3 && (pk_m != 8 || key == 3);
    if (rows_only || ksel > 2 || metric != VD_METRIC_EUCLID || (pk_mode == 0 && !first_ok))
      return vd_fail(VD_EINVAL, "packed pass: step %d, key form %d, layout %d", k, key, pk_m);
    return launch_pass_pk(a, grid, block, nb, pk_m, ksel, pk_mode, dedup, st, pdl);
  }
  // a pass over a row range (one band of a split map) always takes the plain kernel
  if (!rows_only && sparse && ksel <= 2)
    return launch_pass_sparse(a, grid, block, nb, metric, key, ksel, dedup, st, pdl);
  // the shared-memory tiled form: opt-in (tile_max_k > 0).  It stages one
  // table read per tile pixel instead of one per candidate, but its tile takes
  // most of the SM's L1, so with large tables (2^18 seeds: 1 MB) the staging
  // reads go to L2 behind a block barrier: on the GB300, 8192^2 with 2^18
  // seeds, k = 2 234 -> 333 us and k = 8 274 -> 435 us; with 2^14 seeds
  // (64 KB table) k <= 2 about even
  if (!rows_only && tile_max_k > 0 && tile_applies(k, key, tile_max_k))
    return launch_pass_tile(a, nb, key, tile_rows, st, pdl);
  // the register-blocked form: opt-in (blocked == 1).  It loads and gathers
  // each vector once for up to four quads, but needs 64 registers a thread
  // (half the resident warps) and measured slower than the plain pass on the
  // GB300 (8192^2, 2^18 seeds: Von Neumann k = 32 189 -> 244 us, Moore k = 8
  // 268 -> 275 us; 2^14 seeds likewise), so auto leaves it off
  if (!rows_only && blocked == 1 && blk_applies(k, key))
    return launch_pass_blk(a, nb, key, dedup, key_pack, blk_min_blocks, st, pdl);
  cudaError_t e;
  if (nb == VD_NB_MOORE) {
    if (metric == VD_METRIC_EUCLID) {
      e = key == 4 ? launch_pass_t<vdk::kMoore, vdk::kEuclid, 4>(ksel, dedup, grid, block, st, pdl, a)
          : key == 3 ? launch_pass_t<vdk::kMoore, vdk::kEuclid, 3>(ksel, dedup, grid, block, st, pdl, a)
          : key    ? launch_pass_t<vdk::kMoore, vdk::kEuclid, 1>(ksel, dedup, grid, block, st, pdl, a)
                   : launch_pass_t<vdk::kMoore, vdk::kEuclid, 0>(ksel, dedup, grid, block, st, pdl, a);
    } else {
      e = key == 2 ? launch_pass_t<vdk::kMoore, vdk::kManhattan, 2>(ksel, dedup, grid, block, st, pdl, a)
          : key    ? launch_pass_t<vdk::kMoore, vdk::kManhattan, 1>(ksel, dedup, grid, block, st, pdl, a)
                   : launch_pass_t<vdk::kMoore, vdk::kManhattan, 0>(ksel, dedup, grid, block, st, pdl, a);
    }
  } else {
    if (metric == VD_METRIC_EUCLID) {
      e = key == 4 ? launch_pass_t<vdk::kVonNeumann, vdk::kEuclid, 4>(ksel, dedup, grid, block, st, pdl, a)
          : key == 3 ? launch_pass_t<vdk::kVonNeumann, vdk::kEuclid, 3>(ksel, dedup, grid, block, st, pdl, a)
          : key    ? launch_pass_t<vdk::kVonNeumann, vdk::kEuclid, 1>(ksel, dedup, grid, block, st, pdl, a)
                   : launch_pass_t<vdk::kVonNeumann, vdk::kEuclid, 0>(ksel, dedup, grid, block, st, pdl, a);
    } else {
      e = key == 2 ? launch_pass_t<vdk::kVonNeumann, vdk::kManhattan, 2>(ksel, dedup, grid, block, st, pdl, a)
          : key    ? launch_pass_t<vdk::kVonNeumann, vdk::kManhattan, 1>(ksel, dedup, grid, block, st, pdl, a)
                   : launch_pass_t<vdk::kVonNeumann, vdk::kManhattan, 0>(ksel, dedup, grid, block, st, pdl, a);
    }
  }
  if (e != cudaSuccess) return vd_cuda_check(e, "jump pass launch");
  return vd_cuda_check(cudaGetLastError(), "jump pass launch");
}

int launch_fused(const MapView& m, const int32_t* src, int32_t* dst, const int32_t* ks,
                 const int32_t* nbs, int n, int32_t metric, int tile_x, int tile_y,
                 cudaStream_t st) {
  static size_t smem_done[2] = {0, 0};
  vdk::FusedArgs a;
  std::memset(&a, 0, sizeof(a));
  a.src = src;
  a.dst = dst;
  a.table = m.table;
  a.n_seeds = static_cast<uint32_t>(m.n);
  a.w = m.w;
  a.h = m.h;
  a.pitch = m.pitch;
  a.n_pass = n;
  a.halo = 0;
  for (int i = 0; i < n; ++i) {
    a.ks[i] = ks[i];
    a.nbs[i] = nbs[i];
    a.halo += ks[i];
  }
  a.tx = tile_x;
  a.ty = tile_y;
  const size_t smem =
      2ull * (tile_x + 2 * a.halo) * (tile_y + 2 * a.halo) * sizeof(int32_t);
  dim3 block(32, 8);
  dim3 grid((m.w + tile_x - 1) / tile_x, (m.h + tile_y - 1) / tile_y);
  int rc;
  if (metric == VD_METRIC_EUCLID) {
    rc = ensure_smem(reinterpret_cast<const void*>(&vdk::k_pass_fused<vdk::kEuclid>), smem, &smem_done[0]);
    if (rc) return rc;
    vdk::k_pass_fused<vdk::kEuclid><<<grid, block, smem, st>>>(a);
  } else {
    rc = ensure_smem(reinterpret_cast<const void*>(&vdk::k_pass_fused<vdk::kManhattan>), smem, &smem_done[1]);
    if (rc) return rc;
    vdk::k_pass_fused<vdk::kManhattan><<<grid, block, smem, st>>>(a);
  }
  return vd_cuda_check(cudaGetLastError(), "fused pass launch");
}

// Splits a frame's passes into launches: large steps one launch each, runs of
// steps <= fuse_max_k into shared-memory groups (a lone small pass stays
// unfused).  Returns the launch plan.
std::vector<Launch> plan_passes(const int32_t* ks, const int32_t* nbs, int n, int fuse_max_k,
                                int max_halo) {
  std::vector<Launch> plan;
  int i = 0;
  while (i < n) {
    if (fuse_max_k <= 0 || ks[i] > fuse_max_k) {
      Launch l;
      l.n = 1;
      l.first = i;
      plan.push_back(l);
      ++i;
      continue;
    }
    int j = i, halo = 0;
    while (j < n && ks[j] <= fuse_max_k && j - i < vdk::kMaxFused && halo + ks[j] <= max_halo) {
      halo += ks[j];
      ++j;
    }
    Launch l;
    l.first = i;
    l.n = j - i;
    plan.push_back(l);
    i = j;
  }
  return plan;
}

bool use_sparse(int sparse_option, int32_t w, int32_t h, int32_t n, int32_t k) {
  if (sparse_option >= 0) return sparse_option == 1;
  // auto: k <= c / 32 with c = sqrt(w h / n), the mean cell side, where
  // nearly every quad lies inside one cell with all its candidates.  The
  // block-wide test and compaction cost about 0.45 of a plain pass when no
  // quad is unchanged (its second reading of the labels misses L1), so it
  // only pays from about 85% unchanged quads on (GB300, 8192^2: 2^14 seeds,
  // k = 1, 87% unchanged: 217 -> 200 us; k = 4, 66%: 256 -> 276 us; 2^10
  // seeds, D = 1: dJFA frame 2.50 -> 2.38 ms)
  return 1024.0 * k * k * static_cast<double>(n) <= static_cast<double>(w) * h;
}

int run_passes(const MapView& m, int32_t* const buf[2], int* cur, const int32_t* ks,
               const int32_t* nbs, int n, int32_t metric, const Tuning& t, cudaStream_t st,
               int64_t* launches, Profiler* prof, bool djfa_frame) {
  const std::vector<Launch> plan = plan_passes(ks, nbs, n, t.fuse_max_k, t.max_halo);
  const int64_t px = static_cast<int64_t>(m.w) * m.h;
  // the frame's last passes on position-tagged words: [pk_first, n), at least
  // two of them (the first reads the plain map, the last writes it), never
  // with shared-memory fusion
  int pk_first = n;
  const int pk_m = t.fuse_max_k <= 0 ? pk_bits(m.n) : 0;
  if (pk_m) {
    while (pk_first > 0 && use_packed(t, metric, m.w, m.h, m.n, ks[pk_first - 1], ks[0], djfa_frame)) --pk_first;
    if (n - pk_first < 2) pk_first = n;
  }
  for (const Launch& l : plan) {
    const int32_t* src = buf[*cur];
    int32_t* dst = buf[*cur ^ 1];
    int rc;
    const int pi = prof ? prof->begin(l.n == 1 ? VD_KERNEL_PASS : VD_KERNEL_FUSED, px * l.n, st) : -1;
    if (l.n == 1) {
      rc = launch_pass(m, src, dst, ks[l.first], nbs[l.first], metric, t.band_min_k,
                       use_clamp(t.clamp, metric, m.n, ks[l.first], djfa_frame), st, t.pdl != 0,
                       use_dedup(t.dedup, m.w, m.h, m.n, djfa_frame),
                       use_byte_key(t.byte_key, metric, m.w, m.h, m.n, ks[l.first], djfa_frame), t.blocked,
                       t.key_pack, t.blk_min_blocks,
                       use_sparse(t.sparse, m.w, m.h, m.n, ks[l.first]), 0, -1, t.pass_bx, t.tile_max_k,
                       t.tile_rows, l.first >= pk_first ? pk_m : 0,
                       l.first == pk_first ? 0 : (l.first == n - 1 ? 2 : 1));
    } else {
      rc = launch_fused(m, src, dst, ks + l.first, nbs + l.first, l.n, metric, t.tile_x, t.tile_y, st);
    }
    if (prof) prof->end(pi, st);
    if (rc) return rc;
    ++*launches;
    *cur ^= 1;
  }
  return VD_OK;
}

bool use_packed(const Tuning& t, int32_t metric, int32_t w, int32_t h, int32_t n, int32_t k, int32_t k_first,
                bool djfa_frame) {
  if (t.packed == 0 || !djfa_frame || metric != VD_METRIC_EUCLID) return false;
  const int lay = pk_bits(n);
  if (lay == 0 || !(k == 1 || k == 2 || k % 4 == 0)) return false;
  // the split layout's first pass folds with the clamped key, the others'
  // with the byte-offset key
  if (!(lay == 4 ? use_clamp(t.clamp, metric, n, k, djfa_frame) : use_byte_key(t.byte_key, metric, w, h, n, k,
                                                                               djfa_frame)))
    return false;
  if (t.packed == 1) return true;
  // auto: the byte-offset key's bounds (mean cell radius at most 40 pixels
  // per 128 of window, k at most twice the window) with the layout's window
  const double hw = static_cast<double>(1 << (lay - 1));
  if (k > 2 * hw) return false;
  // The split layout's +-8 window: after a frame's first step of 16 (moves
  // of more than 8 pixels) the map is still that far off two passes later.
  // Estimated on the CPU at 16 pixels a seed (1024^2, 2^16 seeds), the share
  // of quads whose winner fails the check in the first pass on words: first
  // step 8, that pass at k = 4: 0.05% (moves of 1), 0.65% (4); first step
  // 16, at k = 8: 85%, at k = 4: 26%, at k = 2: 0.12%.  So words from
  // k * first step <= 64 on, i.e. the words passes start two steps after a
  // first step of 16 and right after one of 8
  if (lay == 4 && static_cast<int64_t>(k) * k_first > 64) return false;
  const double r_max = 40.0 * hw / 128.0;
  return static_cast<double>(w) * h <= 3.141592653589793 * r_max * r_max * n;
}

bool use_dedup(int dedup_option, int32_t w, int32_t h, int32_t n, bool djfa_frame) {
  if (dedup_option >= 0) return dedup_option == 1;
  // auto: dJFA passes on maps of at most 256 pixels per seed.  There most
  // quads straddle a cell boundary and the table outgrows L1, so skipping a
  // repeated gather saves more than the compares cost; in JFA frames (many
  // empty and changing labels) and with larger cells it loses.
  return djfa_frame && static_cast<int64_t>(w) * h <= 256 * static_cast<int64_t>(n);
}

static int grid1d(int64_t n, int block) { return static_cast<int>((n + block - 1) / block); }

int launch_fill(int32_t* buf, int64_t n_elems, int32_t v, cudaStream_t st) {
  const int64_t n4 = n_elems / 4;
  int blocks = grid1d(n4, 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  vdk::k_fill<<<blocks, 256, 0, st>>>(reinterpret_cast<int4*>(buf), n4, v);
  return vd_cuda_check(cudaGetLastError(), "fill launch");
}

int launch_stamp(const MapView& m, int32_t* labels, bool mark, cudaStream_t st, int64_t* launches, bool pdl) {
  const int blocks = grid1d(m.n, 256);
  // one kernel: on a map with stale labels (mark) the swap-and-restore
  // stamp, on an emptied one the atomic minimum alone; either may start
  // while its predecessor drains, and writes the frame's seed entries of the
  // wide and split position-tagged layouts
  const int pkm = pk_bits(m.n) == 8 ? 0 : pk_bits(m.n);
  const cudaError_t e = launch_k(mark ? vdk::k_stamp_xchg : vdk::k_stamp_min, dim3(blocks), dim3(256), st, pdl,
                                 labels, m.pitch, m.seeds, m.n, pkm ? m.pkf : nullptr, m.ptable - 1, pkm);
  if (e != cudaSuccess) return vd_cuda_check(e, "stamp launch");
  ++*launches;
  return vd_cuda_check(cudaGetLastError(), "stamp launch");
}

int launch_move(int2* seeds, int2* table, uint32_t* ptable, int n, const int2* dxy, int w, int h, int max_disp,
                uint64_t key, uint64_t step, cudaStream_t st) {
  vdk::MoveArgs a;
  a.seeds = seeds;
  a.table = table;
  a.ptable = ptable;
  a.n = n;
  a.dxy = dxy;
  a.w = w;
  a.h = h;
  a.max_disp = max_disp;
  a.key = key;
  a.step = step;
  vdk::k_move<<<grid1d(n, 256), 256, 0, st>>>(a);
  return vd_cuda_check(cudaGetLastError(), "move launch");
}

int launch_build_table(const int2* seeds, int n, int2* table, uint32_t* ptable, cudaStream_t st) {
  vdk::k_build_table<<<grid1d(n, 256), 256, 0, st>>>(seeds, n, table, ptable);
  return vd_cuda_check(cudaGetLastError(), "table launch");
}

uint64_t rng_key(uint64_t rng_seed, uint64_t stream_id) { return vdk::splitmix64(rng_seed, stream_id); }

cudaEvent_t Profiler::take() {
  if (!spare.empty()) {
    cudaEvent_t e = spare.back();
    spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

int Profiler::begin(int kind, int64_t u, cudaStream_t st) {
  Rec r;
  r.kind = kind;
  r.units = u;
  r.a = take();
  r.b = take();
  if (!r.a || !r.b) return -1;
  cudaEventRecord(r.a, st);
  pending.push_back(r);
  return static_cast<int>(pending.size()) - 1;
}

void Profiler::end(int idx, cudaStream_t st) {
  if (idx >= 0) cudaEventRecord(pending[idx].b, st);
}

int Profiler::collect(cudaStream_t st) {
  const int rc = vd_cuda_check(cudaStreamSynchronize(st), "synchronize");
  if (rc) return rc;
  for (const Rec& r : pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      ms[r.kind] += t;
      launches[r.kind] += 1;
      units[r.kind] += r.units;
    } else {
      cudaGetLastError();
    }
    spare.push_back(r.a);
    spare.push_back(r.b);
  }
  pending.clear();
  return VD_OK;
}

void Profiler::reset() {
  for (const Rec& r : pending) {
    spare.push_back(r.a);
    spare.push_back(r.b);
  }
  pending.clear();
  for (int i = 0; i < 8; ++i) {
    ms[i] = 0;
    launches[i] = 0;
    units[i] = 0;
  }
}

void Profiler::destroy() {
  reset();
  for (cudaEvent_t e : spare) cudaEventDestroy(e);
  spare.clear();
}

}  // namespace vdi

// ---------------------------------------------------------------------------
// The context
// ---------------------------------------------------------------------------

struct vd_ctx {
  int device = 0;
  int32_t w = 0, h = 0, n = 0, pitch = 0;
  int32_t cap = 0;       // seeds the seed-sized buffers hold (>= n)
  bool repair = false;   // seeds were removed: the next dJFA frame runs the repair schedule
  cudaStream_t stream = nullptr;
  int32_t* buf[2] = {nullptr, nullptr};
  int cur = 0;
  int2* pbuf[2] = {nullptr, nullptr};  // position maps of JFA frames (allocated on first use)
  int2* seeds = nullptr;
  int2* table = nullptr;   // n + 1 entries, [0] = sentinel
  uint32_t* ptable = nullptr;  // n + 1 packed positions, [0] = far position
  uint2* pkf = nullptr;        // n + 1 entries of the position-tagged passes, [0] = far position
  int2* dxy_stage = nullptr;
  // vd_step's host displacements: two device buffers (capacity dxy_in_cap)
  // filled on h2d_stream while the previous step computes
  int2* dxy_in[2] = {nullptr, nullptr};
  int dxy_in_cap = 0;
  int dxy_next = 0;
  cudaStream_t h2d_stream = nullptr;
  cudaEvent_t dxy_ready[2] = {nullptr, nullptr};
  cudaEvent_t dxy_free[2] = {nullptr, nullptr};
  unsigned long long* counters = nullptr;      // [0] n_exact, [1] n_match, [2] flag
  unsigned long long* host_counters = nullptr;  // pinned mirror
  int32_t* stage_a = nullptr;  // dense w*h staging (exact distances / exact labels)
  int32_t* stage_b = nullptr;  // dense w*h staging (reference labels / exact distances)
  // bucket grid of vd_exact
  int* bk_count = nullptr;
  int* bk_start = nullptr;
  int* bk_ids = nullptr;
  int64_t bk_cells = 0;
  // asynchronous label read-back: two snapshot slots copied out on copy_stream
  int32_t* snap[2] = {nullptr, nullptr};
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t snap_ready[2] = {nullptr, nullptr};
  cudaEvent_t copy_done[2] = {nullptr, nullptr};
  bool copy_pending[2] = {false, false};
  int snap_next = 0;
  vdi::Tuning tune;
  vdi::Profiler prof;
  int64_t launches = 0;
  // captured frames: the executable graph, and for a whole step the graph and
  // its move node, whose arguments change every call
  struct FrameGraph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t move = nullptr;
  };
  std::map<std::tuple<int, int, int, int, int, int, int>, FrameGraph> graphs;
};

static vdi::Profiler* prof_of(vd_ctx* c) { return c->tune.profile ? &c->prof : nullptr; }

static void clear_graphs(vd_ctx* c) {
  for (auto& kv : c->graphs) {
    cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  c->graphs.clear();
}

static vdi::MapView view(const vd_ctx* c) {
  vdi::MapView m;
  m.w = c->w;
  m.h = c->h;
  m.pitch = c->pitch;
  m.n = c->n;
  m.seeds = c->seeds;
  m.table = c->table + 1;
  m.ptable = c->ptable + 1;
  m.pkf = c->pkf;
  return m;
}

static int ctx_alloc(void** p, size_t bytes, const char* what) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return vd_fail(VD_ENOMEM, "cudaMalloc(%zu bytes) for %s: %s", bytes, what, cudaGetErrorString(e));
  }
  return VD_OK;
}

static void ctx_free(vd_ctx* c) {
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  for (int i = 0; i < 2; ++i) {
    cudaFree(c->snap[i]);
    if (c->snap_ready[i]) cudaEventDestroy(c->snap_ready[i]);
    if (c->copy_done[i]) cudaEventDestroy(c->copy_done[i]);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  c->prof.destroy();
  clear_graphs(c);
  cudaFree(c->buf[0]);
  cudaFree(c->buf[1]);
  cudaFree(c->pbuf[0]);
  cudaFree(c->pbuf[1]);
  cudaFree(c->seeds);
  cudaFree(c->table);
  cudaFree(c->ptable);
  cudaFree(c->pkf);
  cudaFree(c->dxy_stage);
  if (c->h2d_stream) cudaStreamSynchronize(c->h2d_stream);
  for (int i = 0; i < 2; ++i) {
    cudaFree(c->dxy_in[i]);
    if (c->dxy_ready[i]) cudaEventDestroy(c->dxy_ready[i]);
    if (c->dxy_free[i]) cudaEventDestroy(c->dxy_free[i]);
  }
  if (c->h2d_stream) cudaStreamDestroy(c->h2d_stream);
  cudaFree(c->counters);
  cudaFreeHost(c->host_counters);
  cudaFree(c->stage_a);
  cudaFree(c->stage_b);
  cudaFree(c->bk_count);
  cudaFree(c->bk_start);
  cudaFree(c->bk_ids);
}

extern "C" vd_ctx* vd_create(int32_t w, int32_t h, int32_t n) {
  if (bad_side(w) || bad_side(h)) {
    vd_fail(VD_EINVAL, "grid %dx%d outside [1, %d]", w, h, VD_MAX_SIDE);
    return nullptr;
  }
  if (n < 1) {
    vd_fail(VD_EINVAL, "n_seeds %d < 1", n);
    return nullptr;
  }
  vd_ctx* c = new vd_ctx();
  cudaGetDevice(&c->device);
  c->w = w;
  c->h = h;
  c->n = n;
  c->pitch = (w + 31) / 32 * 32;
  c->cap = n;
  const size_t map_bytes = static_cast<size_t>(c->pitch) * h * sizeof(int32_t);
  int rc = VD_OK;
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->buf[0]), map_bytes, "label map");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->buf[1]), map_bytes, "label map");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->seeds), sizeof(int2) * n, "seeds");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->table), sizeof(int2) * (static_cast<size_t>(n) + 1), "seed table");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->ptable), sizeof(uint32_t) * (static_cast<size_t>(n) + 1), "seed table");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->pkf), sizeof(uint2) * (static_cast<size_t>(n) + 1), "seed table");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->dxy_stage), sizeof(int2) * n, "moves");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&c->counters), 4 * sizeof(unsigned long long), "counters");
  if (!rc) {
    const cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&c->host_counters), 4 * sizeof(unsigned long long));
    if (e != cudaSuccess) rc = vd_cuda_check(e, "cudaMallocHost(counters)");
  }
  if (!rc) rc = vd_cuda_check(cudaMemset(c->buf[0], 0xFF, map_bytes), "init map");
  if (!rc) rc = vd_cuda_check(cudaMemset(c->buf[1], 0xFF, map_bytes), "init map");
  if (!rc) rc = vd_cuda_check(cudaMemset(c->seeds, 0, sizeof(int2) * n), "init seeds");
  if (!rc) rc = vdi::launch_build_table(c->seeds, n, c->table, c->ptable, nullptr);
  if (!rc) rc = vd_cuda_check(cudaDeviceSynchronize(), "create");
  if (rc) {
    ctx_free(c);
    delete c;
    return nullptr;
  }
  return c;
}

extern "C" int vd_destroy(vd_ctx* c) {
  if (!c) return VD_OK;
  cudaStreamSynchronize(c->stream);
  ctx_free(c);
  delete c;
  return VD_OK;
}

#define VD_CHECK_CTX(c) \
  if (!(c)) return vd_fail(VD_EINVAL, "null context")

extern "C" int vd_set_stream(vd_ctx* c, void* stream) {
  VD_CHECK_CTX(c);
  c->stream = static_cast<cudaStream_t>(stream);
  clear_graphs(c);
  return VD_OK;
}

extern "C" int vd_synchronize(vd_ctx* c) {
  VD_CHECK_CTX(c);
  return vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
}

extern "C" int vd_get_shape(const vd_ctx* c, int32_t* w, int32_t* h, int32_t* n, int32_t* pitch) {
  VD_CHECK_CTX(c);
  if (w) *w = c->w;
  if (h) *h = c->h;
  if (n) *n = c->n;
  if (pitch) *pitch = c->pitch;
  return VD_OK;
}

static cudaMemcpyKind kind_from(int on_device) {
  return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
}

extern "C" int vd_set_seeds(vd_ctx* c, const int32_t* xy, int on_device) {
  VD_CHECK_CTX(c);
  if (!xy) return vd_fail(VD_EINVAL, "null seeds");
  if (!on_device) {
    for (int32_t k = 0; k < c->n; ++k) {
      const int32_t x = xy[2 * k], y = xy[2 * k + 1];
      if (x < 0 || x >= c->w || y < 0 || y >= c->h)
        return vd_fail(VD_EINVAL, "seed %d at (%d, %d) outside the %dx%d grid", k, x, y, c->w, c->h);
    }
  }
  if (!on_device) {
    const int rc = vd_cuda_check(cudaMemcpyAsync(c->seeds, xy, sizeof(int2) * c->n, cudaMemcpyHostToDevice, c->stream),
                                 "copy seeds");
    if (rc) return rc;
    ++c->launches;
    return vdi::launch_build_table(c->seeds, c->n, c->table, c->ptable, c->stream);
  }
  // device input: validate in the staging buffer so that rejected seeds never
  // reach the kernels that index the map with them
  int rc = vd_cuda_check(cudaMemcpyAsync(c->dxy_stage, xy, sizeof(int2) * c->n, cudaMemcpyDeviceToDevice, c->stream),
                         "copy seeds");
  if (!rc) rc = vd_cuda_check(cudaMemsetAsync(c->counters + 2, 0, sizeof(unsigned long long), c->stream), "memset");
  if (rc) return rc;
  vdk::k_check_seeds<<<(c->n + 255) / 256, 256, 0, c->stream>>>(c->dxy_stage, c->n, c->w, c->h, c->counters + 2);
  ++c->launches;
  rc = vd_cuda_check(cudaGetLastError(), "check seeds");
  if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(c->host_counters + 2, c->counters + 2, sizeof(unsigned long long),
                                              cudaMemcpyDeviceToHost, c->stream), "copy flag");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
  if (rc) return rc;
  if (c->host_counters[2] != 0)
    return vd_fail(VD_EINVAL, "%llu device seeds outside the %dx%d grid", c->host_counters[2], c->w, c->h);
  rc = vd_cuda_check(cudaMemcpyAsync(c->seeds, c->dxy_stage, sizeof(int2) * c->n, cudaMemcpyDeviceToDevice, c->stream),
                     "copy seeds");
  if (rc) return rc;
  ++c->launches;
  return vdi::launch_build_table(c->seeds, c->n, c->table, c->ptable, c->stream);
}

// Seed-sized buffers for `cap` seeds (seeds, both pass tables, staging);
// the old ones are released.  Leaves the context unchanged on failure.
static int grow_seed_buffers(vd_ctx* c, int32_t cap, const int* keep, const int* newidx, const int2* add,
                             int32_t n_add) {
  int2* seeds = nullptr;
  int2* table = nullptr;
  uint32_t* ptable = nullptr;
  uint2* pkf = nullptr;
  int2* stage = nullptr;
  int rc = ctx_alloc(reinterpret_cast<void**>(&seeds), sizeof(int2) * cap, "seeds");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&table), sizeof(int2) * (static_cast<size_t>(cap) + 1), "seed table");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&ptable), sizeof(uint32_t) * (static_cast<size_t>(cap) + 1), "seed table");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&pkf), sizeof(uint2) * (static_cast<size_t>(cap) + 1), "seed table");
  rc = rc ? rc : ctx_alloc(reinterpret_cast<void**>(&stage), sizeof(int2) * cap, "moves");
  if (rc) {
    cudaFree(seeds);
    cudaFree(table);
    cudaFree(ptable);
    cudaFree(pkf);
    cudaFree(stage);
    return rc;
  }
  const int total = c->n + n_add;
  vdk::k_update_compact<<<(total + 255) / 256, 256, 0, c->stream>>>(c->seeds, c->n, keep, newidx, add, n_add, seeds);
  rc = vd_cuda_check(cudaGetLastError(), "compact seeds");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
  if (rc) {
    cudaFree(seeds);
    cudaFree(table);
    cudaFree(ptable);
    cudaFree(pkf);
    cudaFree(stage);
    return rc;
  }
  cudaFree(c->seeds);
  cudaFree(c->table);
  cudaFree(c->ptable);
  cudaFree(c->pkf);
  cudaFree(c->dxy_stage);
  cudaFree(c->bk_ids);  // sized by the seed count; reallocated on next use
  c->bk_ids = nullptr;
  c->seeds = seeds;
  c->table = table;
  c->ptable = ptable;
  c->pkf = pkf;
  c->dxy_stage = stage;
  c->cap = cap;
  return VD_OK;
}

extern "C" int vd_update_seeds(vd_ctx* c, const int32_t* remove_ids, int32_t n_remove, const int32_t* add_xy,
                               int32_t n_add, int on_device) {
  VD_CHECK_CTX(c);
  if (n_remove < 0 || n_add < 0) return vd_fail(VD_EINVAL, "negative counts (%d removed, %d added)", n_remove, n_add);
  if ((n_remove > 0 && !remove_ids) || (n_add > 0 && !add_xy)) return vd_fail(VD_EINVAL, "null input");
  if (n_remove > c->n) return vd_fail(VD_EINVAL, "%d removals of %d seeds", n_remove, c->n);
  const int64_t n_new = static_cast<int64_t>(c->n) - n_remove + n_add;
  if (n_new < 1) return vd_fail(VD_EINVAL, "no seed would remain");
  if (n_new > (int64_t{1} << 30)) return vd_fail(VD_EINVAL, "%lld seeds exceed 2^30", static_cast<long long>(n_new));
  cudaStream_t st = c->stream;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // stream-ordered scratch: keep flags, new indices (+ the survivor count), the inputs
  int* keep = nullptr;
  int* newidx = nullptr;
  int* rem = nullptr;
  int2* add = nullptr;
  auto release = [&]() {
    if (keep) cudaFreeAsync(keep, st);
    if (newidx) cudaFreeAsync(newidx, st);
    if (rem) cudaFreeAsync(rem, st);
    if (add) cudaFreeAsync(add, st);
  };
  int rc = vd_cuda_check(cudaMallocAsync(reinterpret_cast<void**>(&keep), sizeof(int) * c->n, st), "update scratch");
  if (!rc) rc = vd_cuda_check(cudaMallocAsync(reinterpret_cast<void**>(&newidx), sizeof(int) * (c->n + 1), st), "update scratch");
  if (!rc && n_remove > 0) rc = vd_cuda_check(cudaMallocAsync(reinterpret_cast<void**>(&rem), sizeof(int) * n_remove, st), "update scratch");
  if (!rc && n_add > 0) rc = vd_cuda_check(cudaMallocAsync(reinterpret_cast<void**>(&add), sizeof(int2) * n_add, st), "update scratch");
  if (!rc && n_remove > 0) rc = vd_cuda_check(cudaMemcpyAsync(rem, remove_ids, sizeof(int) * n_remove, kind, st), "copy removals");
  if (!rc && n_add > 0) rc = vd_cuda_check(cudaMemcpyAsync(add, add_xy, sizeof(int2) * n_add, kind, st), "copy new seeds");
  if (!rc) rc = vd_cuda_check(cudaMemsetAsync(c->counters + 2, 0, sizeof(unsigned long long), st), "memset");
  if (rc) {
    release();
    return rc;
  }
  // validate first: nothing of the context changes unless every removal
  // names a distinct seed and every new seed lies on the grid.  Host inputs
  // are checked on the host (the update then stays asynchronous); device
  // inputs by the flagging kernels, read back once.
  if (!on_device) {
    std::vector<char> seen(static_cast<size_t>(c->n), 0);
    for (int32_t j = 0; j < n_remove && !rc; ++j) {
      const int32_t id = remove_ids[j];
      if (id < 0 || id >= c->n) rc = vd_fail(VD_EINVAL, "removal %d names seed %d of %d", j, id, c->n);
      else if (seen[id]++) rc = vd_fail(VD_EINVAL, "seed %d removed twice", id);
    }
    for (int32_t j = 0; j < n_add && !rc; ++j) {
      const int32_t x = add_xy[2 * j], y = add_xy[2 * j + 1];
      if (x < 0 || x >= c->w || y < 0 || y >= c->h)
        rc = vd_fail(VD_EINVAL, "new seed %d at (%d, %d) outside the %dx%d grid", j, x, y, c->w, c->h);
    }
    if (rc) {
      release();
      return rc;
    }
  }
  vdk::k_fill_i32<<<std::min((c->n + 255) / 256, 152 * 8), 256, 0, st>>>(keep, c->n, 1);
  if (n_remove > 0)
    vdk::k_update_remove<<<(n_remove + 255) / 256, 256, 0, st>>>(rem, n_remove, c->n, keep, c->counters + 2);
  c->launches += 1 + (n_remove > 0);
  rc = vd_cuda_check(cudaGetLastError(), "validate update");
  if (!rc && on_device) {
    if (n_add > 0) vdk::k_check_seeds<<<(n_add + 255) / 256, 256, 0, st>>>(add, n_add, c->w, c->h, c->counters + 2);
    c->launches += n_add > 0;
    rc = vd_cuda_check(cudaGetLastError(), "validate update");
    if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(c->host_counters + 2, c->counters + 2, sizeof(unsigned long long),
                                                cudaMemcpyDeviceToHost, st), "copy flag");
    if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(st), "synchronize");
    if (!rc && c->host_counters[2] != 0)
      rc = vd_fail(VD_EINVAL, "%llu invalid entries (a removal out of range or repeated, or a new seed off the grid)",
                   c->host_counters[2]);
  }
  if (rc) {
    release();
    return rc;
  }
  vdk::k_scan<<<1, 1024, 0, st>>>(keep, c->n, newidx);
  ++c->launches;
  rc = vd_cuda_check(cudaGetLastError(), "scan");
  // the new seed array, then the map relabelled (it still holds old indices)
  if (!rc && n_new > c->cap) {
    rc = grow_seed_buffers(c, static_cast<int32_t>(n_new), keep, newidx, add, n_add);
  } else if (!rc) {
    const int total = c->n + n_add;
    vdk::k_update_compact<<<(total + 255) / 256, 256, 0, st>>>(c->seeds, c->n, keep, newidx, add, n_add, c->dxy_stage);
    rc = vd_cuda_check(cudaGetLastError(), "compact seeds");
    if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(c->seeds, c->dxy_stage, sizeof(int2) * n_new, cudaMemcpyDeviceToDevice, st),
                                "copy seeds");
  }
  ++c->launches;
  if (rc) {
    release();
    return rc;
  }
  const int64_t count = static_cast<int64_t>(c->pitch) * c->h;
  vdk::k_update_relabel<<<static_cast<int>(std::min<int64_t>((count + 255) / 256, 152 * 16)), 256, 0, st>>>(
      c->buf[c->cur], count, keep, newidx);
  ++c->launches;
  rc = vd_cuda_check(cudaGetLastError(), "relabel");
  release();
  if (rc) return rc;
  c->n = static_cast<int32_t>(n_new);
  if (n_remove > 0) c->repair = true;
  // captured frames hold the old seed count and buffers
  clear_graphs(c);
  ++c->launches;
  return vdi::launch_build_table(c->seeds, c->n, c->table, c->ptable, st);
}

extern "C" int vd_get_seeds(vd_ctx* c, int32_t* xy, int on_device) {
  VD_CHECK_CTX(c);
  if (!xy) return vd_fail(VD_EINVAL, "null output");
  int rc = vd_cuda_check(cudaMemcpyAsync(xy, c->seeds, sizeof(int2) * c->n,
                                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                         c->stream), "copy seeds out");
  if (rc || on_device) return rc;
  return vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
}

extern "C" int vd_move_seeds(vd_ctx* c, const int32_t* dxy, int dxy_on_device, int32_t max_disp,
                             uint64_t rng_seed, uint64_t stream_id, int64_t step) {
  VD_CHECK_CTX(c);
  const int2* d = nullptr;
  if (dxy) {
    if (dxy_on_device) {
      if (reinterpret_cast<uintptr_t>(dxy) % alignof(int2) != 0)
        return vd_fail(VD_EINVAL, "device displacements must be 8-byte aligned");
      d = reinterpret_cast<const int2*>(dxy);
    } else {
      const int rc = vd_cuda_check(cudaMemcpyAsync(c->dxy_stage, dxy, sizeof(int2) * c->n,
                                                   cudaMemcpyHostToDevice, c->stream), "copy moves");
      if (rc) return rc;
      d = c->dxy_stage;
    }
  } else {
    if (max_disp < 0 || max_disp > VD_MAX_SIDE) return vd_fail(VD_EINVAL, "max_disp %d outside [0, %d]", max_disp, VD_MAX_SIDE);
    if (step < 0) return vd_fail(VD_EINVAL, "step %lld < 0", static_cast<long long>(step));
  }
  vdi::Profiler* pr = prof_of(c);
  const int pi = pr ? pr->begin(VD_KERNEL_MOVE, c->n, c->stream) : -1;
  const int rc = vdi::launch_move(c->seeds, c->table, c->ptable, c->n, d, c->w, c->h, max_disp,
                                  vdi::rng_key(rng_seed, stream_id), static_cast<uint64_t>(step), c->stream);
  if (pr) pr->end(pi, c->stream);
  ++c->launches;
  return rc;
}

static int check_metric(int32_t metric) {
  if (metric != VD_METRIC_EUCLID && metric != VD_METRIC_MANHATTAN) return vd_fail(VD_EINVAL, "metric %d", metric);
  return VD_OK;
}

// Runs a frame body either eagerly or as a cached CUDA graph.  `key` must
// identify the launch sequence completely (it includes the buffer parity).
// With `move`, the body's first launch is the move kernel, whose arguments
// (displacements, RNG step) change every call: the graph keeps that node and
// its arguments are replaced before each launch.
template <typename F>
static int run_frame(vd_ctx* c, const std::tuple<int, int, int, int, int, int, int>& key, int n_launch,
                     int cur_after, F&& body, const vdk::MoveArgs* move = nullptr) {
  if (!c->tune.use_graphs || c->tune.profile || c->stream == nullptr) {
    return body();
  }
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    cudaGraph_t g = nullptr;
    int rc = vd_cuda_check(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (rc) return rc;
    const int cur0 = c->cur;
    const int64_t l0 = c->launches;
    const int brc = body();
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    c->cur = cur0;
    c->launches = l0;
    if (brc) {
      if (g) cudaGraphDestroy(g);
      return brc;
    }
    rc = vd_cuda_check(ee, "end capture");
    if (rc) return rc;
    vd_ctx::FrameGraph fg;
    if (move) {
      // the move node: the graph's kernel node running vdk::k_move
      size_t count = 0;
      rc = vd_cuda_check(cudaGraphGetNodes(g, nullptr, &count), "graph nodes");
      std::vector<cudaGraphNode_t> nodes(count);
      if (!rc && count) rc = vd_cuda_check(cudaGraphGetNodes(g, nodes.data(), &count), "graph nodes");
      for (size_t i = 0; !rc && i < count && !fg.move; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p;
        if (cudaGraphKernelNodeGetParams(nodes[i], &p) == cudaSuccess &&
            p.func == reinterpret_cast<void*>(vdk::k_move))
          fg.move = nodes[i];
      }
      if (!rc && !fg.move) rc = vd_fail(VD_ECUDA, "captured step has no move kernel");
      if (rc) {
        cudaGraphDestroy(g);
        return rc;
      }
    }
    rc = vd_cuda_check(cudaGraphInstantiate(&fg.exec, g, 0), "graph instantiate");
    if (rc) {
      cudaGraphDestroy(g);
      return rc;
    }
    if (move) fg.graph = g;  // kept: its move node addresses the executable's copy
    else cudaGraphDestroy(g);
    it = c->graphs.emplace(key, fg).first;
  }
  if (move) {
    cudaKernelNodeParams p{};
    p.func = reinterpret_cast<void*>(vdk::k_move);
    p.gridDim = dim3((c->n + 255) / 256);
    p.blockDim = dim3(256);
    p.sharedMemBytes = 0;
    vdk::MoveArgs a = *move;
    void* args[] = {&a};
    p.kernelParams = args;
    p.extra = nullptr;
    const int rc = vd_cuda_check(cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.move, &p), "step arguments");
    if (rc) return rc;
  }
  const int rc = vd_cuda_check(cudaGraphLaunch(it->second.exec, c->stream), "graph launch");
  if (rc) return rc;
  c->cur = cur_after;
  c->launches += n_launch;
  return VD_OK;
}

static int count_launches(const int32_t* ks, const int32_t* nbs, int n, const vdi::Tuning& t) {
  return static_cast<int>(vdi::plan_passes(ks, nbs, n, t.fuse_max_k, t.max_halo).size());
}

// Leading passes of a JFA schedule that run on the position map (k % 4 == 0,
// k >= 4), or 0 when the position map is not used for this context.
static int jfa_position_passes(const vd_ctx* c, const int32_t* ks, int n) {
  if (c->tune.pos_map == 0) return 0;
  // auto: maps of at least 2^20 pixels (GB300, 8192^2 JFA frames: 2^18 seeds
  // 7.27 -> 4.27 ms, 2^22 seeds 11.96 -> 5.28 ms, 2^14 seeds 4.42 -> 4.12 ms,
  // 2^10 seeds 4.09 -> 4.04 ms)
  if (c->tune.pos_map < 0 && static_cast<int64_t>(c->w) * c->h < (int64_t{1} << 20)) return 0;
  int m = 0;
  while (m < n && ks[m] >= 4 && ks[m] % 4 == 0) ++m;
  return m;
}

extern "C" int vd_jfa(vd_ctx* c, int32_t extra, int32_t metric) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  int32_t ks[VD_MAX_PASSES], nbs[VD_MAX_PASSES];
  const int n = vd_jfa_schedule(c->w, c->h, extra, ks, nbs, VD_MAX_PASSES);
  if (n < 0) return n;
  const int m = jfa_position_passes(c, ks, n);
  if (m > 0 && !c->pbuf[0]) {
    const size_t bytes = sizeof(int2) * static_cast<size_t>(c->pitch) * c->h;
    int rc = ctx_alloc(reinterpret_cast<void**>(&c->pbuf[0]), bytes, "position map");
    if (!rc) rc = ctx_alloc(reinterpret_cast<void**>(&c->pbuf[1]), bytes, "position map");
    if (rc) {
      cudaFree(c->pbuf[0]);
      c->pbuf[0] = c->pbuf[1] = nullptr;
      return rc;
    }
  }
  // launches after the fill and the stamp: the position-map passes (the last
  // of them writes the label map), then the rest on the label map
  const int nl = m > 0 ? m + count_launches(ks + m, nbs + m, n - m, c->tune) : count_launches(ks, nbs, n, c->tune);
  const int flips = m > 0 ? 1 + count_launches(ks + m, nbs + m, n - m, c->tune) : nl;
  const int cur_after = c->cur ^ (flips & 1);
  auto body = [&]() -> int {
    vdi::Profiler* pr = prof_of(c);
    const bool pdl = c->tune.pdl != 0;
    const int64_t px = static_cast<int64_t>(c->w) * c->h;
    if (m > 0) {
      int pi = pr ? pr->begin(VD_KERNEL_FILL, px, c->stream) : -1;
      int rc = vdi::launch_fill_pos(c->pbuf[0], static_cast<int64_t>(c->pitch) * c->h, c->stream, pdl);
      if (pr) pr->end(pi, c->stream);
      ++c->launches;
      if (rc) return rc;
      pi = pr ? pr->begin(VD_KERNEL_STAMP, c->n, c->stream) : -1;
      rc = vdi::launch_stamp_pos(view(c), c->pbuf[0], c->stream, pdl);
      if (pr) pr->end(pi, c->stream);
      ++c->launches;
      if (rc) return rc;
      for (int i = 0; i < m; ++i) {
        const bool last = i == m - 1;
        pi = pr ? pr->begin(VD_KERNEL_PASS, px, c->stream) : -1;
        rc = vdi::launch_pass_pos(view(c), c->pbuf[i & 1], last ? nullptr : c->pbuf[(i + 1) & 1],
                                  last ? c->buf[c->cur ^ 1] : nullptr, ks[i], nbs[i], metric, c->tune.band_min_k,
                                  c->stream, pdl);
        if (pr) pr->end(pi, c->stream);
        ++c->launches;
        if (rc) return rc;
      }
      c->cur ^= 1;
      // the remaining k = 2, 1 (and extra) passes on the label map, with the
      // JFA frame's key choices (with the dJFA ones, byte-offset key and
      // de-duplicated gathers, the 8192^2, 2^18-seed JFA frame measured
      // 4.25 -> 4.35 ms on the GB300)
      return vdi::run_passes(view(c), c->buf, &c->cur, ks + m, nbs + m, n - m, metric, c->tune, c->stream,
                             &c->launches, pr, false);
    }
    int pi = pr ? pr->begin(VD_KERNEL_FILL, px, c->stream) : -1;
    int rc = vdi::launch_fill(c->buf[c->cur], static_cast<int64_t>(c->pitch) * c->h, -1, c->stream);
    if (pr) pr->end(pi, c->stream);
    ++c->launches;
    if (rc) return rc;
    pi = pr ? pr->begin(VD_KERNEL_STAMP, c->n, c->stream) : -1;
    rc = vdi::launch_stamp(view(c), c->buf[c->cur], false, c->stream, &c->launches, pdl);
    if (pr) pr->end(pi, c->stream);
    if (rc) return rc;
    return vdi::run_passes(view(c), c->buf, &c->cur, ks, nbs, n, metric, c->tune, c->stream, &c->launches, pr,
                           false);
  };
  const int rc = run_frame(c, std::make_tuple(0, c->cur, extra, metric, 0, 0, 0), nl + 2, cur_after, body);
  if (!rc) c->repair = false;  // a full frame covers every pixel
  return rc;
}

extern "C" int vd_djfa_step(vd_ctx* c, int32_t d_max, int32_t vn_waves, int32_t extra, int32_t metric) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  int32_t ks[VD_MAX_PASSES], nbs[VD_MAX_PASSES];
  int n = vd_djfa_schedule(c->w, c->h, c->n, d_max, vn_waves, extra, ks, nbs, VD_MAX_PASSES);
  if (n < 0) return n;
  // after a removal: the full JFA schedule on the relabelled map, so that the
  // emptied cells fill from every side whatever their size
  const bool repair = c->repair;
  if (repair) {
    n = vd_jfa_schedule(c->w, c->h, extra, ks, nbs, VD_MAX_PASSES);
    if (n < 0) return n;
  }
  const int nl = count_launches(ks, nbs, n, c->tune);
  const int cur_after = c->cur ^ (nl & 1);
  auto body = [&]() -> int {
    vdi::Profiler* pr = prof_of(c);
    const int pi = pr ? pr->begin(VD_KERNEL_STAMP, c->n, c->stream) : -1;
    const int rc = vdi::launch_stamp(view(c), c->buf[c->cur], true, c->stream, &c->launches, c->tune.pdl != 0);
    if (pr) pr->end(pi, c->stream);
    if (rc) return rc;
    // a repair frame's map is right except in the emptied cells: the key
    // choices of a dJFA frame suit it (a quad that sees only empty labels
    // falls back to the exact key)
    return vdi::run_passes(view(c), c->buf, &c->cur, ks, nbs, n, metric, c->tune, c->stream, &c->launches, pr,
                           true);
  };
  const int rc = run_frame(c, std::make_tuple(1, c->cur, d_max, vn_waves, extra, metric, repair ? 1 : 0), nl + 1,
                           cur_after, body);
  if (!rc) c->repair = false;
  return rc;
}

// The stream, events and two buffers of vd_step's host displacements.
static int ensure_h2d(vd_ctx* c) {
  int rc = VD_OK;
  if (!c->h2d_stream) {
    rc = vd_cuda_check(cudaStreamCreateWithFlags(&c->h2d_stream, cudaStreamNonBlocking), "stream");
    for (int i = 0; i < 2 && !rc; ++i) {
      rc = vd_cuda_check(cudaEventCreateWithFlags(&c->dxy_ready[i], cudaEventDisableTiming), "event");
      if (!rc) rc = vd_cuda_check(cudaEventCreateWithFlags(&c->dxy_free[i], cudaEventDisableTiming), "event");
    }
    if (rc) return rc;
  }
  if (c->dxy_in_cap < c->n) {
    // (every copy into the old buffers was waited for by the compute stream)
    rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
    for (int i = 0; i < 2; ++i) {
      cudaFree(c->dxy_in[i]);
      c->dxy_in[i] = nullptr;
    }
    c->dxy_in_cap = 0;
    for (int i = 0; i < 2 && !rc; ++i)
      rc = ctx_alloc(reinterpret_cast<void**>(&c->dxy_in[i]), sizeof(int2) * static_cast<size_t>(c->cap), "moves");
    if (rc) return rc;
    c->dxy_in_cap = c->cap;
  }
  return VD_OK;
}

extern "C" int vd_step(vd_ctx* c, const int32_t* dxy, int dxy_on_device, int32_t max_disp, uint64_t rng_seed,
                       uint64_t stream_id, int64_t step, int32_t d_max, int32_t vn_waves, int32_t extra,
                       int32_t metric) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  // the move, as vd_move_seeds
  vdk::MoveArgs ma;
  ma.seeds = c->seeds;
  ma.table = c->table;
  ma.ptable = c->ptable;
  ma.n = c->n;
  ma.dxy = nullptr;
  ma.w = c->w;
  ma.h = c->h;
  ma.max_disp = max_disp;
  ma.key = vdi::rng_key(rng_seed, stream_id);
  ma.step = static_cast<uint64_t>(step);
  if (dxy) {
    if (dxy_on_device) {
      if (reinterpret_cast<uintptr_t>(dxy) % alignof(int2) != 0)
        return vd_fail(VD_EINVAL, "device displacements must be 8-byte aligned");
      ma.dxy = reinterpret_cast<const int2*>(dxy);
    } else {
      ma.dxy = c->dxy_stage;
    }
  } else {
    if (max_disp < 0 || max_disp > VD_MAX_SIDE) return vd_fail(VD_EINVAL, "max_disp %d outside [0, %d]", max_disp, VD_MAX_SIDE);
    if (step < 0) return vd_fail(VD_EINVAL, "step %lld < 0", static_cast<long long>(step));
  }
  int32_t ks[VD_MAX_PASSES], nbs[VD_MAX_PASSES];
  int n = vd_djfa_schedule(c->w, c->h, c->n, d_max, vn_waves, extra, ks, nbs, VD_MAX_PASSES);
  if (n < 0) return n;
  const bool repair = c->repair;
  if (repair) {
    n = vd_jfa_schedule(c->w, c->h, extra, ks, nbs, VD_MAX_PASSES);
    if (n < 0) return n;
  }
  // host displacements come in on their own stream into one of two buffers,
  // so that the copy overlaps the previous step instead of following it;
  // the step waits for it, and the copy into a buffer waits for the step
  // that last read it
  int dslot = -1;
  if (dxy && !dxy_on_device) {
    int rc = ensure_h2d(c);
    if (rc) return rc;
    dslot = c->dxy_next;
    c->dxy_next ^= 1;
    rc = vd_cuda_check(cudaStreamWaitEvent(c->h2d_stream, c->dxy_free[dslot], 0), "wait event");
    if (!rc)
      rc = vd_cuda_check(cudaMemcpyAsync(c->dxy_in[dslot], dxy, sizeof(int2) * c->n, cudaMemcpyHostToDevice,
                                         c->h2d_stream),
                         "copy moves");
    if (!rc) rc = vd_cuda_check(cudaEventRecord(c->dxy_ready[dslot], c->h2d_stream), "event");
    if (!rc) rc = vd_cuda_check(cudaStreamWaitEvent(c->stream, c->dxy_ready[dslot], 0), "wait event");
    if (rc) return rc;
    ma.dxy = c->dxy_in[dslot];
  }
  const int nl = count_launches(ks, nbs, n, c->tune);
  const int cur_after = c->cur ^ (nl & 1);
  auto body = [&]() -> int {
    vdi::Profiler* pr = prof_of(c);
    int pi = pr ? pr->begin(VD_KERNEL_MOVE, c->n, c->stream) : -1;
    vdk::k_move<<<(c->n + 255) / 256, 256, 0, c->stream>>>(ma);
    if (pr) pr->end(pi, c->stream);
    ++c->launches;
    int rc = vd_cuda_check(cudaGetLastError(), "move launch");
    if (rc) return rc;
    pi = pr ? pr->begin(VD_KERNEL_STAMP, c->n, c->stream) : -1;
    rc = vdi::launch_stamp(view(c), c->buf[c->cur], true, c->stream, &c->launches, c->tune.pdl != 0);
    if (pr) pr->end(pi, c->stream);
    if (rc) return rc;
    return vdi::run_passes(view(c), c->buf, &c->cur, ks, nbs, n, metric, c->tune, c->stream, &c->launches, pr,
                           true);
  };
  const int rc = run_frame(c, std::make_tuple(2, c->cur, d_max, vn_waves, extra, metric, repair ? 1 : 0), nl + 2,
                           cur_after, body, &ma);
  if (!rc) c->repair = false;
  if (dslot >= 0) {
    const int erc = vd_cuda_check(cudaEventRecord(c->dxy_free[dslot], c->stream), "event");
    if (!rc) return erc;
  }
  return rc;
}

extern "C" int vd_stamp(vd_ctx* c) {
  VD_CHECK_CTX(c);
  return vdi::launch_stamp(view(c), c->buf[c->cur], true, c->stream, &c->launches);
}

extern "C" int vd_pass(vd_ctx* c, int32_t k, int32_t nb, int32_t metric) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  if (k < 1) return vd_fail(VD_EINVAL, "step %d < 1", k);
  if (nb != VD_NB_MOORE && nb != VD_NB_VON_NEUMANN) return vd_fail(VD_EINVAL, "neighbourhood %d", nb);
  const int rc = vdi::launch_pass(view(c), c->buf[c->cur], c->buf[c->cur ^ 1], k, nb, metric,
                                  c->tune.band_min_k, vdi::use_clamp(c->tune.clamp, metric, c->n, k, false),
                                  c->stream, false, vdi::use_dedup(c->tune.dedup, c->w, c->h, c->n, false),
                                  vdi::use_byte_key(c->tune.byte_key, metric, c->w, c->h, c->n, k, false),
                                  c->tune.blocked, c->tune.key_pack, c->tune.blk_min_blocks,
                                  vdi::use_sparse(c->tune.sparse, c->w, c->h, c->n, k), 0, -1, c->tune.pass_bx,
                                  c->tune.tile_max_k, c->tune.tile_rows);
  if (rc) return rc;
  ++c->launches;
  c->cur ^= 1;
  return VD_OK;
}

// Times `steps` dJFA steps (vd_step, RNG moves of steps 0 .. steps - 1) from
// the snapshot with the tuning `t`; returns ms per step in *ms.
struct TuneSnapshot {
  int32_t* map = nullptr;
  int2* seeds = nullptr;
  int2* table = nullptr;
  uint32_t* ptable = nullptr;
  int cur = 0;
  bool repair = false;
  void release() {
    cudaFree(map);
    cudaFree(seeds);
    cudaFree(table);
    cudaFree(ptable);
    map = nullptr;
    seeds = nullptr;
    table = nullptr;
    ptable = nullptr;
  }
};

static int tune_snapshot(vd_ctx* c, TuneSnapshot& sn, bool save) {
  const size_t map_bytes = sizeof(int32_t) * static_cast<size_t>(c->pitch) * c->h;
  const size_t n = static_cast<size_t>(c->n);
  cudaError_t e;
  if (save) {
    sn.cur = c->cur;
    sn.repair = c->repair;
    e = cudaMemcpyAsync(sn.map, c->buf[c->cur], map_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sn.seeds, c->seeds, sizeof(int2) * n, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sn.table, c->table, sizeof(int2) * (n + 1), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(sn.ptable, c->ptable, sizeof(uint32_t) * (n + 1), cudaMemcpyDeviceToDevice, c->stream);
  } else {
    c->cur = sn.cur;
    c->repair = sn.repair;
    e = cudaMemcpyAsync(c->buf[c->cur], sn.map, map_bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->seeds, sn.seeds, sizeof(int2) * n, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->table, sn.table, sizeof(int2) * (n + 1), cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(c->ptable, sn.ptable, sizeof(uint32_t) * (n + 1), cudaMemcpyDeviceToDevice, c->stream);
  }
  return vd_cuda_check(e, "autotune snapshot copy");
}

extern "C" int vd_autotune(vd_ctx* c, int32_t d_max, int32_t max_disp, int32_t vn_waves, int32_t metric,
                           uint64_t rng_seed, int32_t steps, int32_t* chosen, double* ms_per_step, int32_t cap) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  if (steps < 1 || steps > 1000) return vd_fail(VD_EINVAL, "steps outside [1, 1000]");
  if (max_disp < 0 || d_max < 0) return vd_fail(VD_EINVAL, "negative displacement bound");
  if (cap > 0 && !ms_per_step) return vd_fail(VD_EINVAL, "null times with cap > 0");
  int32_t ks[VD_MAX_PASSES], nbs[VD_MAX_PASSES];
  if (vd_djfa_schedule(c->w, c->h, c->n, d_max, vn_waves, 0, ks, nbs, VD_MAX_PASSES) < 0) return VD_EINVAL;
  TuneSnapshot sn;
  const size_t map_bytes = sizeof(int32_t) * static_cast<size_t>(c->pitch) * c->h;
  int rc = ctx_alloc(reinterpret_cast<void**>(&sn.map), map_bytes, "autotune snapshot");
  if (!rc) rc = ctx_alloc(reinterpret_cast<void**>(&sn.seeds), sizeof(int2) * c->n, "autotune snapshot");
  if (!rc) rc = ctx_alloc(reinterpret_cast<void**>(&sn.table), sizeof(int2) * (static_cast<size_t>(c->n) + 1), "autotune snapshot");
  if (!rc) rc = ctx_alloc(reinterpret_cast<void**>(&sn.ptable), sizeof(uint32_t) * (static_cast<size_t>(c->n) + 1), "autotune snapshot");
  if (!rc) rc = tune_snapshot(c, sn, true);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc) rc = vd_cuda_check(cudaEventCreate(&e0), "event");
  if (!rc) rc = vd_cuda_check(cudaEventCreate(&e1), "event");
  const vdi::Tuning t0 = c->tune;
  const int64_t launches0 = c->launches;
  int measured = 0;
  auto measure = [&](const vdi::Tuning& t, double* ms) -> int {
    c->tune = t;
    c->tune.profile = 0;
    clear_graphs(c);
    int r = tune_snapshot(c, sn, false);
    // one untimed step (graph capture), then the timed ones, each from the snapshot
    for (int s = 0; !r && s <= steps; ++s) {
      if (s == 1) r = vd_cuda_check(cudaEventRecord(e0, c->stream), "event");
      if (!r) r = vd_step(c, nullptr, 0, max_disp, rng_seed, 0, s, d_max, vn_waves, 0, metric);
    }
    if (!r) r = vd_cuda_check(cudaEventRecord(e1, c->stream), "event");
    if (!r) r = vd_cuda_check(cudaEventSynchronize(e1), "event sync");
    float el = 0.f;
    if (!r) r = vd_cuda_check(cudaEventElapsedTime(&el, e0, e1), "elapsed");
    if (!r) {
      *ms = static_cast<double>(el) / steps;
      if (ms_per_step && measured < cap) ms_per_step[measured] = *ms;
      ++measured;
    }
    return r;
  };
  // coordinate search: each dimension in turn, the others at the best so far
  vdi::Tuning best = t0;
  double best_ms = 0.0;
  if (!rc) rc = measure(best, &best_ms);
  struct Dim {
    int vdi::Tuning::*field;
    std::vector<int> values;
  };
  const Dim dims[] = {
      {&vdi::Tuning::packed, {-1, 0}},             // position-tagged passes (auto, off)
      {&vdi::Tuning::pass_bx, {64, 32, 128}},      // block tile
      {&vdi::Tuning::dedup, {-1, 0, 1}},           // gather de-duplication
      {&vdi::Tuning::sparse, {-1, 0, 1}},          // sparse form of small steps
      {&vdi::Tuning::blocked, {-1, 1}},            // register-blocked byte-key form
      {&vdi::Tuning::blk_min_blocks, {8, 6}},      // its blocks per SM
      {&vdi::Tuning::fuse_max_k, {0, 2, 4}},       // shared-memory fusion depth of small steps
      {&vdi::Tuning::tile_max_k, {0, 2, 8}},       // shared-memory tiled byte-key passes
      {&vdi::Tuning::tile_rows, {16, 8}},          // and that tile's rows
  };
  for (const Dim& d : dims) {
    if (rc) break;
    if (d.field == &vdi::Tuning::blk_min_blocks && best.blocked != 1) continue;  // no effect
    if (d.field == &vdi::Tuning::tile_rows && best.tile_max_k == 0) continue;      // no effect
    const int start = best.*(d.field);
    for (int v : d.values) {
      if (rc) break;
      if (v == start) continue;
      vdi::Tuning t = best;
      t.*(d.field) = v;
      double ms = 0.0;
      rc = measure(t, &ms);
      if (!rc && ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  }
  // the state exactly as it was, and the fastest setting kept
  const int rrc = tune_snapshot(c, sn, false);
  if (!rc) rc = rrc;
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  sn.release();
  c->tune = rc ? t0 : best;
  c->tune.profile = t0.profile;
  c->tune.use_graphs = t0.use_graphs;
  c->launches = launches0;
  clear_graphs(c);
  if (rc) return rc;
  if (chosen) {
    chosen[0] = best.pass_bx;
    chosen[1] = best.dedup;
    chosen[2] = best.sparse;
    chosen[3] = best.blocked;
    chosen[4] = best.blk_min_blocks;
    chosen[5] = best.fuse_max_k;
    chosen[6] = best.tile_max_k;
    chosen[7] = best.tile_rows;
    chosen[8] = best.packed;
  }
  return measured;
}

extern "C" int vd_pass_rows(vd_ctx* c, int32_t k, int32_t nb, int32_t metric, int32_t y0, int32_t y1,
                            int32_t djfa_frame) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  if (k < 1) return vd_fail(VD_EINVAL, "step %d < 1", k);
  if (nb != VD_NB_MOORE && nb != VD_NB_VON_NEUMANN) return vd_fail(VD_EINVAL, "neighbourhood %d", nb);
  if (y0 < 0 || y1 > c->h || y0 >= y1) return vd_fail(VD_EINVAL, "rows [%d, %d) outside [0, %d)", y0, y1, c->h);
  const bool dj = djfa_frame != 0;
  const int rc = vdi::launch_pass(view(c), c->buf[c->cur], c->buf[c->cur ^ 1], k, nb, metric,
                                  c->tune.band_min_k, vdi::use_clamp(c->tune.clamp, metric, c->n, k, dj),
                                  c->stream, false, vdi::use_dedup(c->tune.dedup, c->w, c->h, c->n, dj),
                                  vdi::use_byte_key(c->tune.byte_key, metric, c->w, c->h, c->n, k, dj), 0, 0, 8,
                                  false, y0, y1, c->tune.pass_bx);
  if (rc) return rc;
  ++c->launches;
  c->cur ^= 1;
  return VD_OK;
}

extern "C" int vd_clear_labels(vd_ctx* c) {
  VD_CHECK_CTX(c);
  const int rc = vdi::launch_fill(c->buf[c->cur], static_cast<int64_t>(c->pitch) * c->h, -1, c->stream);
  if (rc) return rc;
  ++c->launches;
  return VD_OK;
}

extern "C" int vd_set_labels(vd_ctx* c, const int32_t* labels, int on_device) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null labels");
  const int64_t total = static_cast<int64_t>(c->w) * c->h;
  if (!on_device) {
    for (int64_t i = 0; i < total; ++i)
      if (labels[i] < -1 || labels[i] >= c->n)
        return vd_fail(VD_EINVAL, "label %d at %lld outside [-1, %d)", labels[i], static_cast<long long>(i), c->n);
  } else {
    // the passes index the seed table with every label: reject out-of-range
    // device labels before they reach the map
    int rc = vd_cuda_check(cudaMemsetAsync(c->counters + 2, 0, sizeof(unsigned long long), c->stream), "memset");
    if (rc) return rc;
    int blocks = static_cast<int>((total + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    vdk::k_check_labels<<<blocks, 256, 0, c->stream>>>(labels, total, c->n, c->counters + 2);
    ++c->launches;
    rc = vd_cuda_check(cudaGetLastError(), "check labels");
    if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(c->host_counters + 2, c->counters + 2, sizeof(unsigned long long),
                                                cudaMemcpyDeviceToHost, c->stream), "copy flag");
    if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
    if (rc) return rc;
    if (c->host_counters[2] != 0)
      return vd_fail(VD_EINVAL, "%llu device labels outside [-1, %d)", c->host_counters[2], c->n);
  }
  return vd_cuda_check(cudaMemcpy2DAsync(c->buf[c->cur], sizeof(int32_t) * c->pitch, labels, sizeof(int32_t) * c->w,
                                         sizeof(int32_t) * c->w, c->h, kind_from(on_device), c->stream),
                       "copy labels in");
}

extern "C" int vd_get_labels(vd_ctx* c, int32_t* labels, int on_device) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  int rc = vd_cuda_check(cudaMemcpy2DAsync(labels, sizeof(int32_t) * c->w, c->buf[c->cur], sizeof(int32_t) * c->pitch,
                                           sizeof(int32_t) * c->w, c->h,
                                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
                         "copy labels out");
  if (rc || on_device) return rc;
  return vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
}

extern "C" int vd_labels_device_ptr(vd_ctx* c, const int32_t** labels) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  *labels = c->buf[c->cur];
  return VD_OK;
}

static int ensure_stage(vd_ctx* c, int32_t** p) {
  if (*p) return VD_OK;
  return ctx_alloc(reinterpret_cast<void**>(p), sizeof(int32_t) * static_cast<size_t>(c->w) * c->h, "staging map");
}

static int similarity_launch(vd_ctx* c, const int32_t* exact, int exact_pitch, const int32_t* ref, int ref_pitch,
                             int32_t metric, uint64_t* ne, uint64_t* nm) {
  int rc = vd_cuda_check(cudaMemsetAsync(c->counters, 0, 2 * sizeof(unsigned long long), c->stream), "memset");
  if (rc) return rc;
  const int64_t total = static_cast<int64_t>(c->w) * c->h;
  int blocks = static_cast<int>((total + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (metric == VD_METRIC_EUCLID)
    vdk::k_similarity<vdk::kEuclid><<<blocks, 256, 0, c->stream>>>(c->buf[c->cur], c->pitch, c->seeds, c->n, c->w, c->h,
                                                                    exact, exact_pitch, ref, ref_pitch, c->counters);
  else
    vdk::k_similarity<vdk::kManhattan><<<blocks, 256, 0, c->stream>>>(c->buf[c->cur], c->pitch, c->seeds, c->n, c->w,
                                                                       c->h, exact, exact_pitch, ref, ref_pitch, c->counters);
  ++c->launches;
  rc = vd_cuda_check(cudaGetLastError(), "similarity launch");
  if (rc) return rc;
  rc = vd_cuda_check(cudaMemcpyAsync(c->host_counters, c->counters, 2 * sizeof(unsigned long long),
                                     cudaMemcpyDeviceToHost, c->stream), "copy counts");
  if (rc) return rc;
  rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
  if (rc) return rc;
  if (ne) *ne = c->host_counters[0];
  if (nm) *nm = c->host_counters[1];
  return VD_OK;
}

extern "C" int vd_similarity(vd_ctx* c, const int32_t* exact, const int32_t* ref, int on_device, int32_t metric,
                             uint64_t* ne, uint64_t* nm) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  const size_t bytes = sizeof(int32_t) * static_cast<size_t>(c->w) * c->h;
  const int32_t* de = exact;
  const int32_t* dr = ref;
  if (!on_device) {
    if (exact) {
      int rc = ensure_stage(c, &c->stage_a);
      if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(c->stage_a, exact, bytes, cudaMemcpyHostToDevice, c->stream), "copy exact");
      if (rc) return rc;
      de = c->stage_a;
    }
    if (ref) {
      int rc = ensure_stage(c, &c->stage_b);
      if (!rc) rc = vd_cuda_check(cudaMemcpyAsync(c->stage_b, ref, bytes, cudaMemcpyHostToDevice, c->stream), "copy ref");
      if (rc) return rc;
      dr = c->stage_b;
    }
  }
  return similarity_launch(c, de, c->w, dr, c->w, metric, ne, nm);
}

extern "C" int vd_similarity_ctx(vd_ctx* c, vd_ctx* ref, uint64_t* nm) {
  VD_CHECK_CTX(c);
  VD_CHECK_CTX(ref);
  if (ref->w != c->w || ref->h != c->h) return vd_fail(VD_EINVAL, "grid sizes differ");
  if (ref->stream != c->stream) {
    const int rc = vd_cuda_check(cudaStreamSynchronize(ref->stream), "synchronize reference");
    if (rc) return rc;
  }
  return similarity_launch(c, nullptr, 0, ref->buf[ref->cur], ref->pitch, VD_METRIC_EUCLID, nullptr, nm);
}

extern "C" int vd_exact(vd_ctx* c, int32_t* labels, int32_t* dist, int on_device, int32_t metric) {
  VD_CHECK_CTX(c);
  if (check_metric(metric)) return VD_EINVAL;
  // bucket side ~ sqrt(area / seeds): about one seed per bucket
  int cell = 1;
  const double per = static_cast<double>(c->w) * c->h / c->n;
  while (static_cast<double>(cell + 1) * (cell + 1) <= per) ++cell;
  int gw = (c->w + cell - 1) / cell, gh = (c->h + cell - 1) / cell;
  const int64_t cells = static_cast<int64_t>(gw) * gh;
  int rc = VD_OK;
  if (cells > c->bk_cells) {
    cudaFree(c->bk_count);
    cudaFree(c->bk_start);
    c->bk_count = c->bk_start = nullptr;
    c->bk_cells = 0;
    rc = ctx_alloc(reinterpret_cast<void**>(&c->bk_count), sizeof(int) * cells, "bucket counts");
    if (!rc) rc = ctx_alloc(reinterpret_cast<void**>(&c->bk_start), sizeof(int) * (cells + 1), "bucket starts");
    if (rc) return rc;
    c->bk_cells = cells;
  }
  if (!c->bk_ids) rc = ctx_alloc(reinterpret_cast<void**>(&c->bk_ids), sizeof(int) * c->cap, "bucket ids");
  if (rc) return rc;
  int32_t* dl = labels;
  int32_t* dd = dist;
  if (!on_device) {
    if (labels) {
      rc = ensure_stage(c, &c->stage_a);
      if (rc) return rc;
      dl = c->stage_a;
    }
    if (dist) {
      rc = ensure_stage(c, &c->stage_b);
      if (rc) return rc;
      dd = c->stage_b;
    }
  }
  const int sb = (c->n + 255) / 256;
  rc = vd_cuda_check(cudaMemsetAsync(c->bk_count, 0, sizeof(int) * cells, c->stream), "memset");
  if (rc) return rc;
  vdk::k_bucket_count<<<sb, 256, 0, c->stream>>>(c->seeds, c->n, cell, gw, c->bk_count);
  vdk::k_scan<<<1, 1024, 0, c->stream>>>(c->bk_count, static_cast<int>(cells), c->bk_start);
  rc = vd_cuda_check(cudaMemsetAsync(c->bk_count, 0, sizeof(int) * cells, c->stream), "memset");
  if (rc) return rc;
  vdk::k_bucket_fill<<<sb, 256, 0, c->stream>>>(c->seeds, c->n, cell, gw, c->bk_start, c->bk_count, c->bk_ids);
  vdk::Buckets b;
  b.cell = cell;
  b.gw = gw;
  b.gh = gh;
  b.start = c->bk_start;
  b.ids = c->bk_ids;
  dim3 block(32, 8), grid((c->w + 31) / 32, (c->h + 7) / 8);
  if (metric == VD_METRIC_EUCLID)
    vdk::k_exact<vdk::kEuclid><<<grid, block, 0, c->stream>>>(b, c->seeds, c->w, c->h, dl, dd);
  else
    vdk::k_exact<vdk::kManhattan><<<grid, block, 0, c->stream>>>(b, c->seeds, c->w, c->h, dl, dd);
  c->launches += 4;
  rc = vd_cuda_check(cudaGetLastError(), "exact launch");
  if (rc) return rc;
  if (on_device) return VD_OK;
  const size_t bytes = sizeof(int32_t) * static_cast<size_t>(c->w) * c->h;
  if (labels) rc = vd_cuda_check(cudaMemcpyAsync(labels, dl, bytes, cudaMemcpyDeviceToHost, c->stream), "copy out");
  if (!rc && dist) rc = vd_cuda_check(cudaMemcpyAsync(dist, dd, bytes, cudaMemcpyDeviceToHost, c->stream), "copy out");
  if (rc) return rc;
  return vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
}

extern "C" int vd_set_option(vd_ctx* c, int32_t option, int64_t value) {
  VD_CHECK_CTX(c);
  vdi::Tuning t = c->tune;
  switch (option) {
    case VD_OPT_FUSE_MAX_K:
      if (value < 0 || value > 16) return vd_fail(VD_EINVAL, "fuse_max_k %lld outside [0, 16]", static_cast<long long>(value));
      t.fuse_max_k = static_cast<int>(value);
      break;
    case VD_OPT_BAND_ORDER_MIN_K:
      if (value < -1) return vd_fail(VD_EINVAL, "band_min_k %lld < -1", static_cast<long long>(value));
      t.band_min_k = value;
      break;
    case VD_OPT_USE_GRAPHS:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "use_graphs must be 0 or 1");
      t.use_graphs = static_cast<int>(value);
      break;
    case VD_OPT_FUSE_TILE_X:
      if (value < 16 || value > 256 || value % 4) return vd_fail(VD_EINVAL, "tile_x %lld", static_cast<long long>(value));
      t.tile_x = static_cast<int>(value);
      break;
    case VD_OPT_FUSE_TILE_Y:
      if (value < 1 || value > 128) return vd_fail(VD_EINVAL, "tile_y %lld", static_cast<long long>(value));
      t.tile_y = static_cast<int>(value);
      break;
    case VD_OPT_PROFILE:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "profile must be 0 or 1");
      t.profile = static_cast<int>(value);
      break;
    case VD_OPT_CLAMPED_KEYS:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "clamped keys must be -1, 0 or 1");
      t.clamp = static_cast<int>(value);
      break;
    case VD_OPT_PDL:
      if (value != 0 && value != 1) return vd_fail(VD_EINVAL, "pdl must be 0 or 1");
      t.pdl = static_cast<int>(value);
      break;
    case VD_OPT_DEDUP_GATHERS:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "dedup must be -1, 0 or 1");
      t.dedup = static_cast<int>(value);
      break;
    case VD_OPT_BYTE_KEYS:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "byte keys must be -1, 0 or 1");
      t.byte_key = static_cast<int>(value);
      break;
    case VD_OPT_BLOCKED_PASS:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "blocked pass must be -1, 0 or 1");
      t.blocked = static_cast<int>(value);
      break;
    case VD_OPT_KEY_PACK:
      if (value < 0 || value > 2) return vd_fail(VD_EINVAL, "key pack must be 0, 1 or 2");
      t.key_pack = static_cast<int>(value);
      break;
    case VD_OPT_BLOCKED_MIN_BLOCKS:
      if (value != 6 && value != 8) return vd_fail(VD_EINVAL, "blocked-pass blocks per SM must be 6 or 8");
      t.blk_min_blocks = static_cast<int>(value);
      break;
    case VD_OPT_SPARSE_PASS:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "sparse pass must be -1, 0 or 1");
      t.sparse = static_cast<int>(value);
      break;
    case VD_OPT_JFA_POSITION_MAP:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "JFA position map must be -1, 0 or 1");
      t.pos_map = static_cast<int>(value);
      break;
    case VD_OPT_PASS_TILE:
      if (value != 32 && value != 64 && value != 128) return vd_fail(VD_EINVAL, "pass tile must be 32, 64 or 128");
      t.pass_bx = static_cast<int>(value);
      break;
    case VD_OPT_SMEM_TILE_MAX_K:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
        return vd_fail(VD_EINVAL, "shared-memory tile max k must be 0, 1, 2, 4, 8 or 16");
      t.tile_max_k = static_cast<int>(value);
      break;
    case VD_OPT_SMEM_TILE_ROWS:
      if (value != 8 && value != 16) return vd_fail(VD_EINVAL, "shared-memory tile rows must be 8 or 16");
      t.tile_rows = static_cast<int>(value);
      break;
    case VD_OPT_PACKED_MAP:
      if (value < -1 || value > 1) return vd_fail(VD_EINVAL, "packed map must be -1, 0 or 1");
      t.packed = static_cast<int>(value);
      break;
    default:
      return vd_fail(VD_EINVAL, "unknown option %d", option);
  }
  const size_t smem = 2ull * (t.tile_x + 2 * t.max_halo) * (t.tile_y + 2 * t.max_halo) * sizeof(int32_t);
  if (smem > 220 * 1024) return vd_fail(VD_EINVAL, "fused tile needs %zu bytes of shared memory", smem);
  c->tune = t;
  clear_graphs(c);
  return VD_OK;
}

extern "C" int vd_get_option(const vd_ctx* c, int32_t option, int64_t* value) {
  VD_CHECK_CTX(c);
  if (!value) return vd_fail(VD_EINVAL, "null output");
  switch (option) {
    case VD_OPT_FUSE_MAX_K: *value = c->tune.fuse_max_k; break;
    case VD_OPT_BAND_ORDER_MIN_K: *value = c->tune.band_min_k; break;
    case VD_OPT_USE_GRAPHS: *value = c->tune.use_graphs; break;
    case VD_OPT_FUSE_TILE_X: *value = c->tune.tile_x; break;
    case VD_OPT_FUSE_TILE_Y: *value = c->tune.tile_y; break;
    case VD_OPT_PROFILE: *value = c->tune.profile; break;
    case VD_OPT_CLAMPED_KEYS: *value = c->tune.clamp; break;
    case VD_OPT_PDL: *value = c->tune.pdl; break;
    case VD_OPT_DEDUP_GATHERS: *value = c->tune.dedup; break;
    case VD_OPT_BYTE_KEYS: *value = c->tune.byte_key; break;
    case VD_OPT_BLOCKED_PASS: *value = c->tune.blocked; break;
    case VD_OPT_KEY_PACK: *value = c->tune.key_pack; break;
    case VD_OPT_BLOCKED_MIN_BLOCKS: *value = c->tune.blk_min_blocks; break;
    case VD_OPT_SPARSE_PASS: *value = c->tune.sparse; break;
    case VD_OPT_JFA_POSITION_MAP: *value = c->tune.pos_map; break;
    case VD_OPT_PASS_TILE: *value = c->tune.pass_bx; break;
    case VD_OPT_SMEM_TILE_MAX_K: *value = c->tune.tile_max_k; break;
    case VD_OPT_SMEM_TILE_ROWS: *value = c->tune.tile_rows; break;
    case VD_OPT_PACKED_MAP: *value = c->tune.packed; break;
    default: return vd_fail(VD_EINVAL, "unknown option %d", option);
  }
  return VD_OK;
}

extern "C" int64_t vd_launch_count(const vd_ctx* c) { return c ? c->launches : -1; }

extern "C" int vd_profile_read(vd_ctx* c, double* total_ms, int64_t* launches, int64_t* units) {
  VD_CHECK_CTX(c);
  if (!c->tune.profile) return vd_fail(VD_EINVAL, "profiling is off (VD_OPT_PROFILE)");
  const int rc = c->prof.collect(c->stream);
  if (rc) return rc;
  for (int k = 0; k < VD_KERNEL_KINDS; ++k) {
    if (total_ms) total_ms[k] = c->prof.ms[k];
    if (launches) launches[k] = c->prof.launches[k];
    if (units) units[k] = c->prof.units[k];
  }
  return VD_OK;
}

extern "C" int vd_profile_reset(vd_ctx* c) {
  VD_CHECK_CTX(c);
  const int rc = vd_cuda_check(cudaStreamSynchronize(c->stream), "synchronize");
  if (rc) return rc;
  c->prof.reset();
  return VD_OK;
}

// ---------------------------------------------------------------------------
// Exact diagram without any allocation (vd_exact_noalloc)
// ---------------------------------------------------------------------------

// Scratch of vd_exact_noalloc: a u64 error flag at the front (ints 0..63 are
// reserved for it), then the bucket counts, bucket starts and seed ids.  Every
// GPU that loads this library holds the array until the process exits.
static __device__ __align__(256) int g_noalloc_scratch[VD_NOALLOC_SCRATCH_INTS];

namespace {

constexpr int kNoallocHeaderInts = 64;

}  // namespace

extern "C" int vd_exact_noalloc(const int32_t* seeds_xy, int32_t n_seeds, int32_t w, int32_t h, int32_t metric,
                                int32_t* labels, int32_t* dist, void* cuda_stream) {
  if (bad_side(w) || bad_side(h)) return vd_fail(VD_EINVAL, "grid %dx%d outside [1, %d]", w, h, VD_MAX_SIDE);
  if (n_seeds < 1) return vd_fail(VD_EINVAL, "n_seeds %d < 1", n_seeds);
  if (!seeds_xy) return vd_fail(VD_EINVAL, "null seeds");
  if (reinterpret_cast<uintptr_t>(seeds_xy) % alignof(int2) != 0)
    return vd_fail(VD_EINVAL, "seeds must be 8-byte aligned");
  if (!labels && !dist) return vd_fail(VD_EINVAL, "no output map");
  if (check_metric(metric)) return VD_EINVAL;
  // bucket side ~ sqrt(area / seeds), then grown until there are at most two
  // buckets per seed (with side 1 and under 4 pixels a seed the first choice
  // alone would give up to 4): the need is then at most 66 + 5 n ints, so
  // every request of up to 200000 seeds fits, whatever the grid
  int cell = 1;
  const double per = static_cast<double>(w) * h / n_seeds;
  while (static_cast<double>(cell + 1) * (cell + 1) <= per) ++cell;
  int gw = (w + cell - 1) / cell, gh = (h + cell - 1) / cell;
  while (static_cast<int64_t>(gw) * gh > 2 * static_cast<int64_t>(n_seeds)) {
    ++cell;
    gw = (w + cell - 1) / cell;
    gh = (h + cell - 1) / cell;
  }
  const int64_t cells = static_cast<int64_t>(gw) * gh;
  const int64_t need = kNoallocHeaderInts + cells + (cells + 1) + n_seeds;
  if (need > VD_NOALLOC_SCRATCH_INTS)
    return vd_fail(VD_EINVAL,
                   "vd_exact_noalloc: %d seeds on a %dx%d grid need %lld scratch ints (%lld buckets), more than "
                   "the static maximum of %d",
                   n_seeds, w, h, static_cast<long long>(need), static_cast<long long>(cells),
                   VD_NOALLOC_SCRATCH_INTS);

  // the host-side name of the array is only a stand-in, the kernels need its
  // device address: resolved on every call (cheap) for the current device's
  // context, so no address outlives a device reset
  void* p = nullptr;
  int rc = vd_cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(scratch)");
  if (rc) return rc;
  int* base = static_cast<int*>(p);
  unsigned long long* flag = reinterpret_cast<unsigned long long*>(base);
  int* count = base + kNoallocHeaderInts;
  int* start = count + cells;
  int* ids = start + cells + 1;
  const int2* seeds = reinterpret_cast<const int2*>(seeds_xy);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int sb = (n_seeds + 255) / 256;

  // seeds outside the grid would index buckets out of range: reject them first
  rc = vd_cuda_check(cudaMemsetAsync(flag, 0, sizeof(unsigned long long), st), "memset");
  if (rc) return rc;
  vdk::k_check_seeds<<<sb, 256, 0, st>>>(seeds, n_seeds, w, h, flag);
  rc = vd_cuda_check(cudaGetLastError(), "check seeds");
  if (rc) return rc;
  unsigned long long bad = 0;
  rc = vd_cuda_check(cudaMemcpyAsync(&bad, flag, sizeof(bad), cudaMemcpyDeviceToHost, st), "copy flag");
  if (!rc) rc = vd_cuda_check(cudaStreamSynchronize(st), "synchronize");
  if (rc) return rc;
  if (bad) return vd_fail(VD_EINVAL, "%llu seeds outside the %dx%d grid", bad, w, h);

  // the array keeps the previous call's contents: the counts restart at zero
  rc = vd_cuda_check(cudaMemsetAsync(count, 0, sizeof(int) * cells, st), "memset");
  if (rc) return rc;
  vdk::k_bucket_count<<<sb, 256, 0, st>>>(seeds, n_seeds, cell, gw, count);
  vdk::k_scan<<<1, 1024, 0, st>>>(count, static_cast<int>(cells), start);
  rc = vd_cuda_check(cudaMemsetAsync(count, 0, sizeof(int) * cells, st), "memset");
  if (rc) return rc;
  vdk::k_bucket_fill<<<sb, 256, 0, st>>>(seeds, n_seeds, cell, gw, start, count, ids);
  vdk::Buckets b;
  b.cell = cell;
  b.gw = gw;
  b.gh = gh;
  b.start = start;
  b.ids = ids;
  dim3 block(32, 8), grid((w + 31) / 32, (h + 7) / 8);
  if (metric == VD_METRIC_EUCLID)
    vdk::k_exact<vdk::kEuclid><<<grid, block, 0, st>>>(b, seeds, w, h, labels, dist);
  else
    vdk::k_exact<vdk::kManhattan><<<grid, block, 0, st>>>(b, seeds, w, h, labels, dist);
  return vd_cuda_check(cudaGetLastError(), "exact launch");
}

// ---------------------------------------------------------------------------
// Asynchronous label read-back
// ---------------------------------------------------------------------------

static int ensure_async(vd_ctx* c) {
  if (c->copy_stream) return VD_OK;
  const size_t bytes = sizeof(int32_t) * static_cast<size_t>(c->pitch) * c->h;
  int rc = VD_OK;
  for (int i = 0; i < 2 && !rc; ++i) rc = ctx_alloc(reinterpret_cast<void**>(&c->snap[i]), bytes, "label snapshot");
  for (int i = 0; i < 2 && !rc; ++i) {
    rc = vd_cuda_check(cudaEventCreateWithFlags(&c->snap_ready[i], cudaEventDisableTiming), "event");
    if (!rc) rc = vd_cuda_check(cudaEventCreateWithFlags(&c->copy_done[i], cudaEventDisableTiming), "event");
  }
  if (!rc) rc = vd_cuda_check(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "copy stream");
  return rc;
}

extern "C" int vd_get_labels_async(vd_ctx* c, int32_t* labels) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  int rc = ensure_async(c);
  if (rc) return rc;
  const int i = c->snap_next;
  c->snap_next ^= 1;
  if (c->copy_pending[i]) {
    // the slot's previous copy must have left the snapshot before it is reused
    rc = vd_cuda_check(cudaEventSynchronize(c->copy_done[i]), "wait for read-back");
    if (rc) return rc;
    c->copy_pending[i] = false;
  }
  const size_t bytes = sizeof(int32_t) * static_cast<size_t>(c->pitch) * c->h;
  // snapshot the current map on the compute stream (later frames rewrite it)
  rc = vd_cuda_check(cudaMemcpyAsync(c->snap[i], c->buf[c->cur], bytes, cudaMemcpyDeviceToDevice, c->stream),
                     "snapshot labels");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->snap_ready[i], c->stream), "event");
  if (!rc) rc = vd_cuda_check(cudaStreamWaitEvent(c->copy_stream, c->snap_ready[i], 0), "wait event");
  if (!rc)
    rc = vd_cuda_check(cudaMemcpy2DAsync(labels, sizeof(int32_t) * c->w, c->snap[i], sizeof(int32_t) * c->pitch,
                                         sizeof(int32_t) * c->w, c->h, cudaMemcpyDeviceToHost, c->copy_stream),
                       "copy labels out");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->copy_done[i], c->copy_stream), "event");
  if (rc) return rc;
  c->copy_pending[i] = true;
  return VD_OK;
}

// Dense 16-bit copy of a label map (rows of w out of a pitched map): labels
// below 2^16 - 1 as they are, the empty label -1 as 0xFFFF.  One thread per
// pixel of row blockIdx.y.
static __global__ void k_narrow16(const int32_t* __restrict__ src, int pitch, int w, uint16_t* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t y = blockIdx.y;
  if (x < w) dst[y * w + x] = static_cast<uint16_t>(src[y * pitch + x]);
}

extern "C" int vd_get_labels16_async(vd_ctx* c, uint16_t* labels) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  if (c->n > 65535) return vd_fail(VD_EINVAL, "16-bit labels need at most 65535 seeds (have %d)", c->n);
  int rc = ensure_async(c);
  if (rc) return rc;
  const int i = c->snap_next;
  c->snap_next ^= 1;
  if (c->copy_pending[i]) {
    // the slot's previous copy must have left the snapshot before it is reused
    rc = vd_cuda_check(cudaEventSynchronize(c->copy_done[i]), "wait for read-back");
    if (rc) return rc;
    c->copy_pending[i] = false;
  }
  // narrow the current map into the slot on the compute stream (later frames
  // rewrite the map), then copy the dense 16-bit map out on the copy stream
  uint16_t* snap = reinterpret_cast<uint16_t*>(c->snap[i]);
  const dim3 grid((c->w + 255) / 256, c->h);
  k_narrow16<<<grid, 256, 0, c->stream>>>(c->buf[c->cur], c->pitch, c->w, snap);
  rc = vd_cuda_check(cudaGetLastError(), "narrow labels");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->snap_ready[i], c->stream), "event");
  if (!rc) rc = vd_cuda_check(cudaStreamWaitEvent(c->copy_stream, c->snap_ready[i], 0), "wait event");
  const size_t bytes = sizeof(uint16_t) * static_cast<size_t>(c->w) * c->h;
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(labels, snap, bytes, cudaMemcpyDeviceToHost, c->copy_stream),
                       "copy labels out");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->copy_done[i], c->copy_stream), "event");
  if (rc) return rc;
  ++c->launches;
  c->copy_pending[i] = true;
  return VD_OK;
}

// Dense 24-bit copy of a label map (rows of w out of a pitched map): each
// label as three little-endian bytes, the empty label -1 as 0xFFFFFF.  With w
// a multiple of 4 a thread packs four labels of one row into three aligned
// 32-bit words (dense byte offset 3 (y w + x) is then a multiple of 12);
// otherwise it stores the three bytes of one label.
static __global__ void k_narrow24x4(const int32_t* __restrict__ src, int pitch, int w, uint32_t* __restrict__ dst) {
  const int x = 4 * static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
  const int64_t y = blockIdx.y;
  if (x >= w) return;
  const int4 l = *reinterpret_cast<const int4*>(src + y * pitch + x);
  const uint32_t a = static_cast<uint32_t>(l.x) & 0xFFFFFFu, b = static_cast<uint32_t>(l.y) & 0xFFFFFFu;
  const uint32_t c = static_cast<uint32_t>(l.z) & 0xFFFFFFu, d = static_cast<uint32_t>(l.w) & 0xFFFFFFu;
  uint32_t* o = dst + 3 * ((y * w + x) / 4);
  o[0] = a | (b << 24);
  o[1] = (b >> 8) | (c << 16);
  o[2] = (c >> 16) | (d << 8);
}

static __global__ void k_narrow24(const int32_t* __restrict__ src, int pitch, int w, uint8_t* __restrict__ dst) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t y = blockIdx.y;
  if (x >= w) return;
  const uint32_t v = static_cast<uint32_t>(src[y * pitch + x]);
  uint8_t* o = dst + 3 * (y * w + x);
  o[0] = static_cast<uint8_t>(v);
  o[1] = static_cast<uint8_t>(v >> 8);
  o[2] = static_cast<uint8_t>(v >> 16);
}

extern "C" int vd_get_labels24_async(vd_ctx* c, uint8_t* labels) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  if (c->n > 0xFFFFFF) return vd_fail(VD_EINVAL, "24-bit labels need at most 16777215 seeds (have %d)", c->n);
  int rc = ensure_async(c);
  if (rc) return rc;
  const int i = c->snap_next;
  c->snap_next ^= 1;
  if (c->copy_pending[i]) {
    // the slot's previous copy must have left the snapshot before it is reused
    rc = vd_cuda_check(cudaEventSynchronize(c->copy_done[i]), "wait for read-back");
    if (rc) return rc;
    c->copy_pending[i] = false;
  }
  // pack the current map into the slot on the compute stream (later frames
  // rewrite the map), then copy the dense 24-bit map out on the copy stream
  if (c->w % 4 == 0) {
    const dim3 grid((c->w / 4 + 255) / 256, c->h);
    k_narrow24x4<<<grid, 256, 0, c->stream>>>(c->buf[c->cur], c->pitch, c->w, reinterpret_cast<uint32_t*>(c->snap[i]));
  } else {
    const dim3 grid((c->w + 255) / 256, c->h);
    k_narrow24<<<grid, 256, 0, c->stream>>>(c->buf[c->cur], c->pitch, c->w, reinterpret_cast<uint8_t*>(c->snap[i]));
  }
  rc = vd_cuda_check(cudaGetLastError(), "pack labels");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->snap_ready[i], c->stream), "event");
  if (!rc) rc = vd_cuda_check(cudaStreamWaitEvent(c->copy_stream, c->snap_ready[i], 0), "wait event");
  const size_t bytes = 3 * static_cast<size_t>(c->w) * c->h;
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(labels, c->snap[i], bytes, cudaMemcpyDeviceToHost, c->copy_stream),
                       "copy labels out");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->copy_done[i], c->copy_stream), "event");
  if (rc) return rc;
  ++c->launches;
  c->copy_pending[i] = true;
  return VD_OK;
}

// Dense bit-packed copy of a label map (rows of w out of a pitched map):
// label j = y w + x occupies bits [j b, (j + 1) b) of a little-endian stream
// of 32-bit words, the empty label -1 as 2^b - 1.  A thread packs 32
// consecutive labels into b words (32 b bits), staged in shared memory so
// that the block's words leave in coalesced stores; words past the stream's
// end (ceil(w h b / 32)) are not written.
constexpr int kPackThreads = 128;
static __global__ void __launch_bounds__(kPackThreads)
    k_pack_bits(const int32_t* __restrict__ src, int pitch, int w, int h, int bits, uint32_t* __restrict__ dst,
                int64_t words) {
  __shared__ uint32_t sm[kPackThreads * 32];
  const int64_t n = static_cast<int64_t>(w) * h;
  const int64_t j0 = (static_cast<int64_t>(blockIdx.x) * kPackThreads + threadIdx.x) * 32;
  const uint32_t mask = bits >= 32 ? 0xFFFFFFFFu : (1u << bits) - 1u;
  uint32_t v[32];
  if (j0 < n && w % 32 == 0) {
    // the 32 labels lie in one row (x is a multiple of 32), in 16-byte vectors
    const int64_t y = j0 / w;
    const int4* p = reinterpret_cast<const int4*>(src + y * pitch + (j0 - y * w));
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int4 t = __ldg(p + q);
      v[4 * q] = static_cast<uint32_t>(t.x);
      v[4 * q + 1] = static_cast<uint32_t>(t.y);
      v[4 * q + 2] = static_cast<uint32_t>(t.z);
      v[4 * q + 3] = static_cast<uint32_t>(t.w);
    }
  } else {
    int64_t y = 0;
    int x = 0;
    if (j0 < n) {
      y = j0 / w;
      x = static_cast<int>(j0 - y * w);
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      v[i] = j0 + i < n ? static_cast<uint32_t>(__ldg(src + y * pitch + x)) : 0u;
      if (++x == w) {
        x = 0;
        ++y;
      }
    }
  }
  uint32_t* s = sm + threadIdx.x * bits;
  unsigned long long acc = 0;
  int have = 0, o = 0;
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    acc |= static_cast<unsigned long long>(v[i] & mask) << have;
    have += bits;
    if (have >= 32) {
      s[o++] = static_cast<uint32_t>(acc);
      acc >>= 32;
      have -= 32;
    }
  }
  __syncthreads();
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kPackThreads * bits;
  for (int i = threadIdx.x; i < kPackThreads * bits; i += kPackThreads)
    if (base + i < words) dst[base + i] = sm[i];
}

extern "C" int vd_get_labels_packed_async(vd_ctx* c, uint8_t* labels, int32_t bits) {
  VD_CHECK_CTX(c);
  if (!labels) return vd_fail(VD_EINVAL, "null output");
  if (bits < 1 || bits > 32) return vd_fail(VD_EINVAL, "label width %d outside [1, 32]", bits);
  if (bits < 32 && static_cast<int64_t>(c->n) > (int64_t{1} << bits) - 1)
    return vd_fail(VD_EINVAL, "%d-bit labels need at most %lld seeds (have %d)", bits,
                   static_cast<long long>((int64_t{1} << bits) - 1), c->n);
  int rc = ensure_async(c);
  if (rc) return rc;
  const int i = c->snap_next;
  c->snap_next ^= 1;
  if (c->copy_pending[i]) {
    rc = vd_cuda_check(cudaEventSynchronize(c->copy_done[i]), "wait for read-back");
    if (rc) return rc;
    c->copy_pending[i] = false;
  }
  // pack the current map into the slot on the compute stream (later frames
  // rewrite the map), then copy the stream out on the copy stream
  const int64_t n = static_cast<int64_t>(c->w) * c->h;
  const int64_t words = (n * bits + 31) / 32;
  const int64_t blocks = ((n + 31) / 32 + kPackThreads - 1) / kPackThreads;
  k_pack_bits<<<static_cast<unsigned>(blocks), kPackThreads, 0, c->stream>>>(
      c->buf[c->cur], c->pitch, c->w, c->h, bits, reinterpret_cast<uint32_t*>(c->snap[i]), words);
  rc = vd_cuda_check(cudaGetLastError(), "pack labels");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->snap_ready[i], c->stream), "event");
  if (!rc) rc = vd_cuda_check(cudaStreamWaitEvent(c->copy_stream, c->snap_ready[i], 0), "wait event");
  const size_t bytes = static_cast<size_t>((n * bits + 7) / 8);
  if (!rc)
    rc = vd_cuda_check(cudaMemcpyAsync(labels, c->snap[i], bytes, cudaMemcpyDeviceToHost, c->copy_stream),
                       "copy labels out");
  if (!rc) rc = vd_cuda_check(cudaEventRecord(c->copy_done[i], c->copy_stream), "event");
  if (rc) return rc;
  ++c->launches;
  c->copy_pending[i] = true;
  return VD_OK;
}

extern "C" int vd_wait_labels(vd_ctx* c) {
  VD_CHECK_CTX(c);
  for (int i = 0; i < 2; ++i) {
    if (!c->copy_pending[i]) continue;
    const int rc = vd_cuda_check(cudaEventSynchronize(c->copy_done[i]), "wait for read-back");
    if (rc) return rc;
    c->copy_pending[i] = false;
  }
  return VD_OK;
}
