// vd_internal.h -- host-side helpers shared by the translation units of the
// CUDA library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

// Records a message for vd_last_error() and returns `code`.
int vd_fail(int code, const char* fmt, ...);
// VD_OK, or VD_ENOMEM / VD_ECUDA with the CUDA error text recorded.
int vd_cuda_check(cudaError_t e, const char* what);

namespace vdi {

// Threads per block of a position-tagged pass (vd_pass_pk.cuh): 256 for the
// Von Neumann passes on words, whose short-lived 128-thread blocks kept only
// 61% of the warp slots filled (8192^2, 2^18 seeds, k = 16: 141 -> 129 us);
// 128 for the rest (the first pass 200 -> 206 us and the Moore passes
// 1-2 us slower at 256).
constexpr int pk_threads(int nb, int mode) { return mode != 0 && nb == 1 ? 256 : 128; }

// What a jump pass needs to know about one map.
struct MapView {
  int32_t w = 0, h = 0, pitch = 0, n = 0;
  const int2* seeds = nullptr;
  const int2* table = nullptr;   // packed pass table, entry -1 = sentinel
  const uint32_t* ptable = nullptr;  // packed positions x | y << 16, entry -1 = far position
  uint2* pkf = nullptr;  // n + 1 entries for the position-tagged passes, [0] = far position
};

// Bits of the largest label (ceil(log2 n_seeds)); clamped 32-bit keys need
// lb >= 4, so that the far sentinel lies beyond the cap 2^(32 - lb) - 1.
int label_bits(int32_t n_seeds);
// Whether a pass with step k uses the clamped key form.
bool use_clamp(int clamp_option, int32_t metric, int32_t n_seeds, int32_t k, bool djfa_frame);

// Launch-shape choices of the jump passes.
struct Tuning {
  int fuse_max_k = 0;     // steps <= this run in shared-memory groups (0 = none)
  int max_halo = 32;      // largest sum of steps in one group
  int64_t band_min_k = -1;  // -1 auto, 0 never, else from this step up
  int use_graphs = 0;
  int tile_x = 64;
  int tile_y = 32;
  int profile = 0;
  int clamp = -1;  // clamped 32-bit keys: -1 auto, 0 never, 1 whenever usable
  int pdl = 1;     // chain a frame's kernels with programmatic dependent launch
  int dedup = -1;  // skip repeated table gathers in a label vector: -1 auto, 0 never, 1 always
  int byte_key = -1;  // Euclidean byte-offset keys: -1 auto, 0 never, 1 whenever usable
  int blocked = -1;   // byte-key passes with k % 4 == 0 register-blocked over 2 x 2 quads: -1 auto, 0, 1
  int key_pack = 0;   // byte-key packing: 0 multiply-add, 1 byte permute (below 2^16 seeds), 2 shift (wide form)
  int blk_min_blocks = 8;  // register budget of the blocked pass: 6 or 8 resident blocks per SM
  int sparse = -1;    // unchanged quads copied through, the rest compacted per block: -1 auto, 0, 1
  int pos_map = -1;   // JFA frames' k % 4 == 0 passes on a (label, position) map: -1 auto, 0, 1
  int pass_bx = 64;   // pass block tile: quads per row (32, 64, 128) x 128 / that many rows
  int tile_max_k = 0;  // byte-key passes with k <= this over a shared-memory tile (0 = never)
  int tile_rows = 16;  // rows of that tile (8 or 16)
  int packed = -1;     // dJFA frames' last byte-key passes on position-tagged words: -1 auto, 0, 1
};

// Event pairs bracketing kernel launches (profiling mode).  Records are kept
// until read; events are recycled afterwards.
struct Profiler {
  struct Rec {
    int kind;
    int64_t units;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> spare;
  double ms[8] = {0};
  int64_t launches[8] = {0};
  int64_t units[8] = {0};
  cudaEvent_t take();
  // Records the opening event of a launch of `kind`; returns its index.
  int begin(int kind, int64_t units, cudaStream_t st);
  void end(int idx, cudaStream_t st);
  int collect(cudaStream_t st);  // synchronises and folds pending records in
  void reset();
  void destroy();
};

// One launch of a frame's plan: passes [first, first + n).
struct Launch {
  int first = 0;
  int n = 0;
};

int ceil_log2(int64_t v);
int32_t jfa_first_step(int32_t w, int32_t h);
int32_t djfa_first_step(int32_t w, int32_t h, int64_t s, int32_t d_max);
int fill_schedule(int32_t first, int32_t vn_waves, int32_t extra, int32_t* ks, int32_t* nbs,
                  int32_t cap);

std::vector<Launch> plan_passes(const int32_t* ks, const int32_t* nbs, int n, int fuse_max_k,
                                int max_halo);
int launch_pass(const MapView& m, const int32_t* src, int32_t* dst, int32_t k, int32_t nb,
                int32_t metric, int64_t band_min_k, bool clamp, cudaStream_t st, bool pdl = false,
                bool dedup = false, bool byte_key = false, int blocked = 0, int key_pack = 0,
                int blk_min_blocks = 8, bool sparse = false, int32_t y0 = 0, int32_t y1 = -1,
                int pass_bx = 64, int tile_max_k = 0, int tile_rows = 16, int pk_m = 0, int pk_mode = 0);
// Whether a pass with step k runs in the sparse form (auto: k at most 1/32 of
// the mean cell side).
bool use_sparse(int sparse_option, int32_t w, int32_t h, int32_t n, int32_t k);
bool use_dedup(int dedup_option, int32_t w, int32_t h, int32_t n, bool djfa_frame);
int byte_key_window(int64_t n, int* lb_out);
bool use_byte_key(int byte_option, int32_t metric, int32_t w, int32_t h, int32_t n, int32_t k,
                  bool djfa_frame);
int launch_fused(const MapView& m, const int32_t* src, int32_t* dst, const int32_t* ks,
                 const int32_t* nbs, int n, int32_t metric, int tile_x, int tile_y,
                 cudaStream_t st);
int run_passes(const MapView& m, int32_t* const buf[2], int* cur, const int32_t* ks,
               const int32_t* nbs, int n, int32_t metric, const Tuning& t, cudaStream_t st,
               int64_t* launches, Profiler* prof, bool djfa_frame);
int launch_fill(int32_t* buf, int64_t n_elems, int32_t v, cudaStream_t st);
int launch_stamp(const MapView& m, int32_t* labels, bool mark, cudaStream_t st, int64_t* launches,
                 bool pdl = false);
int launch_move(int2* seeds, int2* table, uint32_t* ptable, int n, const int2* dxy, int w, int h, int max_disp,
                uint64_t key, uint64_t step, cudaStream_t st);
int launch_build_table(const int2* seeds, int n, int2* table, uint32_t* ptable, cudaStream_t st);
uint64_t rng_key(uint64_t rng_seed, uint64_t stream_id);
int ensure_smem(const void* fn, size_t bytes, size_t* done);

}  // namespace vdi

namespace vdk {
struct PassArgs;
}

namespace vdi {
// The register-blocked byte-key pass (vd_pass_blk.cu): usable for steps
// k % 4 == 0, k >= 4 with the byte-offset key forms (key 3 and 4).
bool blk_applies(int32_t k, int key);
int launch_pass_blk(const vdk::PassArgs& a, int32_t nb, int key, bool dedup, int pack, int minb, cudaStream_t st,
                    bool pdl);
// The sparse pass (vd_pass_sparse.cu): steps with k % 4 == 0, k = 1 or k = 2
// (ksel 0, 1, 2), every key form, the plain pass's launch shape.
int launch_pass_sparse(const vdk::PassArgs& a, dim3 grid, dim3 block, int32_t nb, int32_t metric, int key, int ksel,
                       bool dedup, cudaStream_t st, bool pdl);
// The shared-memory tiled byte-key pass (vd_pass_tile.cu): k = 1, 2 or a
// multiple of 4 up to 16, key forms 3 and 4, at most tile_max_k.
bool tile_applies(int32_t k, int key, int max_k);
int launch_pass_tile(const vdk::PassArgs& a, int32_t nb, int key, int rows, cudaStream_t st, bool pdl);
// The position-tagged dJFA passes (vd_pass_pk.cuh): the word layout M for n
// seeds (8, 7, 6 or 4; 0 where none holds the labels), whether a frame whose
// first step is k_first runs its pass of step k on words, and one pass with step
// k = 1, 2 or k % 4 == 0 (ksel 1, 2, 0) of layout m: mode 0 plain map in,
// words out; 1 words in and out; 2 words in, plain labels out.
int pk_bits(int32_t n);
bool use_packed(const Tuning& t, int32_t metric, int32_t w, int32_t h, int32_t n, int32_t k, int32_t k_first,
                bool djfa_frame);
int launch_pass_pk(const vdk::PassArgs& a, dim3 grid, dim3 block, int32_t nb, int m, int ksel, int mode,
                   bool dedup, cudaStream_t st, bool pdl);
// The position map of JFA frames (vd_pass_pos.cu): per pixel (label, x | y << 16).
int launch_fill_pos(int2* map, int64_t elems, cudaStream_t st, bool pdl);
int launch_stamp_pos(const MapView& m, int2* map, cudaStream_t st, bool pdl);
// One pass with k % 4 == 0 from the position map `src` into `dst`, or, when
// dst32 is set, into that label map.
int launch_pass_pos(const MapView& m, const int2* src, int2* dst, int32_t* dst32, int32_t k, int32_t nb,
                    int32_t metric, int64_t band_min_k, cudaStream_t st, bool pdl);
}  // namespace vdi
