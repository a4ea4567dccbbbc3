// vd_pass_tile.cu -- byte-key passes with small steps over a shared-memory tile.
//
// A pass (Table I for Moore, Section V-B for Von Neumann) scores, for every
// pixel, the seeds named at it and at its neighbours k away.  The plain pass
// gathers one seed-table entry per candidate label (up to nine a pixel); for
// small k neighbouring pixels share most candidates, so here each block of
// 256 x 16 pixels first stages its tile and a k-pixel halo in shared memory as
// (label, packed seed position) pairs -- one table gather per staged pixel,
// about 2 a pixel at k = 8 -- and then reads every candidate with one aligned
// 16-byte shared-memory load per two pixels.  Candidates, the byte-offset key,
// the winner check and its recomputation by the clamped form (vdk::Quad8,
// vdk::byte_fallback) are those of the plain pass; a staged pixel outside the
// map holds the empty label with the far position, whose key, should it win,
// fails the winner check, so every result is exactly the plain pass's.
#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace vdk {

constexpr int kTileQuads = 64;  // 256 pixels a row
constexpr int kTileMaxCols = 5;  // staged columns a thread: (256 + 2 k) / 64, k <= 16

// The byte form's winner check for one quad, then its store (or its
// recomputation by the clamped form); as the tail of pass_quad_byte.
template <int NB, int KSEL, bool WIDE, class Q>
__device__ __forceinline__ void tile_finish(const PassArgs& a, const Q& q, int x0, int y) {
  const uint32_t* __restrict__ arena = a.ptable - 1;
  constexpr uint32_t h = kByteWindow;
  const uint32_t mask = WIDE ? a.bmul - 1u : 0xFFFFu;
  const uint32_t wmask = WIDE ? a.bwin_mask : (0xFFFFu & ~(2u * h - 1u)) * 0x10001u;
  const uint32_t kw = (WIDE ? a.bwin_bias : h * 0x10001u) -
                      (static_cast<uint32_t>(x0) + (static_cast<uint32_t>(y) << 16));
  uint32_t bad = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t j = (q.b[i] + 1u) & mask;
    bad |= (__ldg(&arena[j]) + kw - static_cast<uint32_t>(i)) & wmask;
  }
  const uint32_t top = max(max(q.b[0], q.b[1]), max(q.b[2], q.b[3]));
  if (bad != 0 || top >= (WIDE ? a.blim : (h * h) << 16)) {
    byte_fallback<NB, KSEL, false, false>(a, x0, y);
    return;
  }
  store_quad(a, x0, y, static_cast<int>(q.b[0] & mask), static_cast<int>(q.b[1] & mask),
             static_cast<int>(q.b[2] & mask), static_cast<int>(q.b[3] & mask));
}

// Staged entries e[0 .. 2n) of one row segment, two per 16-byte load.
template <int N>
__device__ __forceinline__ void tile_row(const int2* __restrict__ T, int at, int2 (&e)[N]) {
#pragma unroll
  for (int j = 0; j < N; j += 2) {
    const int4 v = *reinterpret_cast<const int4*>(T + at + j);
    e[j] = make_int2(v.x, v.y);
    e[j + 1] = make_int2(v.z, v.w);
  }
}

// Folds one candidate entry (label, position) into pixel i of the quad.
template <class Q>
__device__ __forceinline__ void tile_fold(Q& q, int i, const int2& e) {
  q.fold(i, make_int2(e.y, 0), e.x);
}

// TR: rows of the tile (16: 1024 threads, 2 blocks an SM; 8: 512, 4).
template <int NB, int KSEL, bool WIDE, int TR>
__global__ void __launch_bounds__(kTileQuads* TR, 2048 / (kTileQuads * TR)) k_pass_tile(PassArgs a) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ int4 tile_smem[];
  int2* T = reinterpret_cast<int2*>(tile_smem);
  const int k = a.k;
  const int RW = 4 * kTileQuads + 2 * k;  // staged pixels a row
  const int RH = TR + 2 * k;
  const int X0 = 4 * kTileQuads * static_cast<int>(blockIdx.x);
  const int Y0 = TR * static_cast<int>(blockIdx.y);
  const int tx = static_cast<int>(threadIdx.x), ty = static_cast<int>(threadIdx.y);
  const uint32_t far = __ldg(&a.ptable[-1]);
  // each staged row: every label load of the thread in flight, then every
  // table read, then the shared-memory stores
  for (int r = ty; r < RH; r += TR) {
    const int gy = Y0 - k + r;
    const bool row_in = gy >= 0 && gy < a.h;
    const int32_t* row = a.src + static_cast<int64_t>(row_in ? gy : 0) * a.pitch;
    int l[kTileMaxCols];
#pragma unroll
    for (int j = 0; j < kTileMaxCols; ++j) {
      const int gx = X0 - k + tx + kTileQuads * j;
      const bool in = row_in && tx + kTileQuads * j < RW && gx >= 0 && gx < a.pitch;
      l[j] = in ? __ldg(row + gx) : -2;  // -2: outside the map (or past the staged row)
    }
    uint32_t e[kTileMaxCols];
#pragma unroll
    for (int j = 0; j < kTileMaxCols; ++j) e[j] = l[j] >= -1 ? __ldg(&a.ptable[l[j]]) : far;
#pragma unroll
    for (int j = 0; j < kTileMaxCols; ++j) {
      const int c = tx + kTileQuads * j;
      if (c < RW) T[r * RW + c] = make_int2(l[j] >= -1 ? l[j] : -1, static_cast<int>(e[j]));
    }
  }
  __syncthreads();
  const int x0 = X0 + 4 * tx, y = Y0 + ty;
  if (x0 >= a.pitch || y >= a.h) return;
  Quad8<false, false, !WIDE && KSEL != 0> q(a, x0, y);
  const int rc = ty + k;  // staged row of y
  if (KSEL == 0) {
    // pixel i takes element i of each neighbouring 4-pixel vector
    const int cc = 4 * tx + k;  // staged column of x0
    int2 e[4];
    tile_row<4>(T, rc * RW + cc, e);
#pragma unroll
    for (int i = 0; i < 4; ++i) q.set(i, make_int2(e[i].y, 0), e[i].x);
#pragma unroll
    for (int dr = -1; dr <= 1; ++dr) {
#pragma unroll
      for (int dc = -1; dc <= 1; ++dc) {
        if ((dr == 0 && dc == 0) || (NB == kVonNeumann && dr != 0 && dc != 0)) continue;
        tile_row<4>(T, (rc + dr * k) * RW + cc + dc * k, e);
#pragma unroll
        for (int i = 0; i < 4; ++i) tile_fold(q, i, e[i]);
      }
    }
  } else {
    // k = 1: staged columns x0 - 1 .. x0 + 4 of a row; pixel i takes
    // columns i - 1, i, i + 1 of it.  k = 2: columns x0 - 2 .. x0 + 5, pixel
    // i takes i - 2, i, i + 2.
    constexpr int N = KSEL == 1 ? 6 : 8;
    int2 e[N];
    tile_row<N>(T, rc * RW + 4 * tx, e);
#pragma unroll
    for (int i = 0; i < 4; ++i) q.set(i, make_int2(e[i + KSEL].y, 0), e[i + KSEL].x);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      tile_fold(q, i, e[i]);
      tile_fold(q, i, e[i + 2 * KSEL]);
    }
#pragma unroll
    for (int dr = -1; dr <= 1; dr += 2) {
      tile_row<N>(T, (rc + dr * k) * RW + 4 * tx, e);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        tile_fold(q, i, e[i + KSEL]);
        if (NB == kMoore) {
          tile_fold(q, i, e[i]);
          tile_fold(q, i, e[i + 2 * KSEL]);
        }
      }
    }
  }
  tile_finish<NB, KSEL, WIDE>(a, q, x0, y);
}

}  // namespace vdk

namespace vdi {

template <int NB, int KSEL, bool WIDE, int TR>
static int launch_tile_t(const vdk::PassArgs& a, cudaStream_t st, bool pdl) {
  static size_t done = 0;
  const size_t smem = sizeof(int2) * static_cast<size_t>(TR + 2 * a.k) * (4 * vdk::kTileQuads + 2 * a.k);
  const int rc = ensure_smem(reinterpret_cast<const void*>(&vdk::k_pass_tile<NB, KSEL, WIDE, TR>), smem, &done);
  if (rc) return rc;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((a.pitch + 4 * vdk::kTileQuads - 1) / (4 * vdk::kTileQuads), (a.h + TR - 1) / TR);
  cfg.blockDim = dim3(vdk::kTileQuads, TR);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, vdk::k_pass_tile<NB, KSEL, WIDE, TR>, a);
  if (e != cudaSuccess) return vd_cuda_check(e, "tiled jump pass launch");
  return vd_cuda_check(cudaGetLastError(), "tiled jump pass launch");
}

bool tile_applies(int32_t k, int key, int max_k) {
  return (key == 3 || key == 4) && k <= max_k && (k == 1 || k == 2 || (k % 4 == 0 && k <= 16));
}

int launch_pass_tile(const vdk::PassArgs& a, int32_t nb, int key, int rows, cudaStream_t st, bool pdl) {
  const int ksel = a.k % 4 == 0 ? 0 : a.k;
  const bool wide = key == 4;
#define VD_TILE_CASE(NBV, KS)                                                                        \
  if (nb == (NBV == vdk::kMoore ? VD_NB_MOORE : VD_NB_VON_NEUMANN) && ksel == KS) {                  \
    if (rows == 8)                                                                                   \
      return wide ? launch_tile_t<NBV, KS, true, 8>(a, st, pdl) : launch_tile_t<NBV, KS, false, 8>(a, st, pdl); \
    return wide ? launch_tile_t<NBV, KS, true, 16>(a, st, pdl) : launch_tile_t<NBV, KS, false, 16>(a, st, pdl); \
  }
  VD_TILE_CASE(vdk::kMoore, 0)
  VD_TILE_CASE(vdk::kMoore, 1)
  VD_TILE_CASE(vdk::kMoore, 2)
  VD_TILE_CASE(vdk::kVonNeumann, 0)
  VD_TILE_CASE(vdk::kVonNeumann, 1)
  VD_TILE_CASE(vdk::kVonNeumann, 2)
#undef VD_TILE_CASE
  return vd_fail(VD_EINVAL, "tiled pass: step %d", a.k);
}

}  // namespace vdi
