// vd_pass_sparse.cu -- the jump pass with unchanged quads copied through and
// the remaining work compacted within each block.
//
// A pass (Table I for Moore, Section V-B for Von Neumann) gives pixel q the
// nearest of the seeds named at q and at its in-grid neighbours q + o k.  When
// every such candidate of a pixel names the pixel's own seed, the pass leaves
// the pixel as it is; when that holds for all four pixels of a thread's quad,
// the quad is copied through without gathering or scoring anything.  Deep
// inside large cells (small k against the cell size) most quads are like
// that, but they are scattered, so a plain per-thread branch would leave most
// warps waiting for the few lanes that do work.  Here each block first tests its quads
// (label loads and XORs only), writes the unchanged ones, and collects the
// rest in shared memory; its threads then score those one per lane with the
// same per-quad code as the plain pass (vdk::pass_quad*).  Every result is
// exactly the plain pass's.
#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace vdk {

// True when every in-grid candidate of each pixel of the quad (x0 .. x0+3, y)
// carries that pixel's own label (then the pass leaves the quad unchanged);
// `own` receives the quad's labels.  Candidates in the row padding read -1
// and make the test fail for a labelled pixel, which only sends the quad to
// the full computation.
template <int NB, int KSEL>
__device__ __forceinline__ bool quad_unchanged(const PassArgs& a, int x0, int y, int4& own) {
  const int64_t pitch = a.pitch;
  const int k = a.k;
  const int32_t* crow = a.src + y * pitch;
  own = __ldg(reinterpret_cast<const int4*>(crow + x0));
  uint32_t acc = 0;
#pragma unroll
  for (int dr = -1; dr <= 1; ++dr) {
    const int yr = y + dr * k;
    if (yr < 0 || yr >= a.h) continue;  // out-of-grid rows hold no candidate
    const int32_t* row = a.src + yr * pitch;
    const bool sides = NB == kMoore || dr == 0;
    if (KSEL == 0) {
      // pixel i takes element i of each neighbouring vector
      if (dr != 0) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(row + x0));
        acc |= (v.x ^ own.x) | (v.y ^ own.y) | (v.z ^ own.z) | (v.w ^ own.w);
      }
      if (sides) {
        if (x0 - k >= 0) {
          const int4 v = __ldg(reinterpret_cast<const int4*>(row + x0 - k));
          acc |= (v.x ^ own.x) | (v.y ^ own.y) | (v.z ^ own.z) | (v.w ^ own.w);
        }
        if (x0 + k < a.pitch) {
          const int4 v = __ldg(reinterpret_cast<const int4*>(row + x0 + k));
          acc |= (v.x ^ own.x) | (v.y ^ own.y) | (v.z ^ own.z) | (v.w ^ own.w);
        }
      }
    } else if (KSEL == 1) {
      // neighbouring pixels are candidates of each other: one label for all
      const int A = own.x;
      if (dr == 0) acc |= (own.y ^ A) | (own.z ^ A) | (own.w ^ A);
      else {
        const int4 v = __ldg(reinterpret_cast<const int4*>(row + x0));
        acc |= (v.x ^ A) | (v.y ^ A) | (v.z ^ A) | (v.w ^ A);
      }
      if (sides) {
        const int l = x0 >= 4 ? __ldg(row + x0 - 1) : A;
        const int r = x0 + 4 < a.pitch ? __ldg(row + x0 + 4) : A;
        acc |= (l ^ A) | (r ^ A);
      }
    } else {
      // k = 2: columns of equal parity are candidates of each other
      const int A = own.x, B = own.y;
      if (dr == 0) acc |= (own.z ^ A) | (own.w ^ B);
      else {
        const int4 v = __ldg(reinterpret_cast<const int4*>(row + x0));
        acc |= (v.x ^ A) | (v.y ^ B) | (v.z ^ A) | (v.w ^ B);
      }
      if (sides) {
        const int2 l = x0 >= 4 ? __ldg(reinterpret_cast<const int2*>(row + x0 - 2)) : make_int2(A, B);
        const int2 r = x0 + 4 < a.pitch ? __ldg(reinterpret_cast<const int2*>(row + x0 + 4)) : make_int2(A, B);
        acc |= (l.x ^ A) | (l.y ^ B) | (r.x ^ A) | (r.y ^ B);
      }
    }
  }
  return acc == 0;
}

template <int NB, int METRIC, int KSEL, int KEY, bool DEDUP>
__device__ __forceinline__ void pass_quad_any(const PassArgs& a, int x0, int y) {
  if (KEY == 3 || KEY == 4) pass_quad_byte<NB, KSEL, false, DEDUP, KEY == 4>(a, x0, y);
  else if (KEY != 0) pass_quad_clamped<NB, KSEL, false, METRIC, DEDUP, KEY == 2>(a, x0, y);
  else pass_quad<NB, METRIC, KSEL, false, DEDUP>(a, x0, y);
}

// Same launch shape and thread -> quad map as k_pass.  The byte-offset forms
// get 40 registers (12 blocks per SM) instead of the plain pass's 32: the
// test and the compaction add live state, which at 32 registers spills.
#ifndef VD_SPARSE_BYTE_MIN_BLOCKS
#define VD_SPARSE_BYTE_MIN_BLOCKS 12
#endif
template <int NB, int METRIC, int KSEL, int KEY, bool DEDUP>
__global__ void __launch_bounds__(kPassThreads, KEY >= 3 ? VD_SPARSE_BYTE_MIN_BLOCKS : VD_PASS_MIN_BLOCKS)
    k_pass_sparse(PassArgs a) {
  pdl_trigger();
  pdl_wait();
  __shared__ int s_n;
  __shared__ uint8_t s_list[kPassThreads];
  const int bx = static_cast<int>(blockDim.x);
  const int tid = static_cast<int>(threadIdx.y) * bx + static_cast<int>(threadIdx.x);
  if (tid == 0) s_n = 0;
  __syncthreads();
  int rb = blockIdx.y;
  if (a.band_m > 1) rb = (blockIdx.y % a.band_t) * a.band_m + blockIdx.y / a.band_t;
  const int xb = 4 * static_cast<int>(blockIdx.x) * bx;
  const int yb = rb * static_cast<int>(blockDim.y);
  const int x0 = xb + 4 * static_cast<int>(threadIdx.x);
  const int y = yb + static_cast<int>(threadIdx.y);
  bool todo = false;
  if (x0 < a.pitch && y < a.h) {
    int4 own;
    if (quad_unchanged<NB, KSEL>(a, x0, y, own)) store_quad(a, x0, y, own.x, own.y, own.z, own.w);
    else todo = true;
  }
  // warp-aggregated append of the quads left to score
  const unsigned m = __ballot_sync(0xFFFFFFFFu, todo);
  const int lane = tid & 31;
  int base = 0;
  if (lane == 0 && m != 0u) base = atomicAdd(&s_n, __popc(m));
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  if (todo) s_list[base + __popc(m & ((1u << lane) - 1u))] = static_cast<uint8_t>(tid);
  __syncthreads();
  const int n = s_n;
  for (int j = tid; j < n; j += kPassThreads) {
    const int t = s_list[j];
    const int ty = t / bx;
    pass_quad_any<NB, METRIC, KSEL, KEY, DEDUP>(a, xb + 4 * (t - ty * bx), yb + ty);
  }
}

}  // namespace vdk

namespace vdi {

static_assert(vdk::kPassThreads <= 256, "thread ids of a block are kept as bytes");

template <int NB, int METRIC, int KSEL, int KEY>
static cudaError_t launch_sparse_t(bool dedup, dim3 g, dim3 b, cudaStream_t st, bool pdl, const vdk::PassArgs& a) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  if (dedup) return cudaLaunchKernelEx(&cfg, vdk::k_pass_sparse<NB, METRIC, KSEL, KEY, true>, a);
  return cudaLaunchKernelEx(&cfg, vdk::k_pass_sparse<NB, METRIC, KSEL, KEY, false>, a);
}

template <int NB, int METRIC, int KEY>
static cudaError_t launch_sparse_k(int ksel, bool dedup, dim3 g, dim3 b, cudaStream_t st, bool pdl,
                                   const vdk::PassArgs& a) {
  switch (ksel) {
    case 0: return launch_sparse_t<NB, METRIC, 0, KEY>(dedup, g, b, st, pdl, a);
    case 1: return launch_sparse_t<NB, METRIC, 1, KEY>(dedup, g, b, st, pdl, a);
    default: return launch_sparse_t<NB, METRIC, 2, KEY>(dedup, g, b, st, pdl, a);
  }
}

template <int NB>
static cudaError_t launch_sparse_nb(int32_t metric, int key, int ksel, bool dedup, dim3 g, dim3 b, cudaStream_t st,
                                    bool pdl, const vdk::PassArgs& a) {
  if (metric == VD_METRIC_EUCLID) {
    switch (key) {
      case 4: return launch_sparse_k<NB, vdk::kEuclid, 4>(ksel, dedup, g, b, st, pdl, a);
      case 3: return launch_sparse_k<NB, vdk::kEuclid, 3>(ksel, dedup, g, b, st, pdl, a);
      case 0: return launch_sparse_k<NB, vdk::kEuclid, 0>(ksel, dedup, g, b, st, pdl, a);
      default: return launch_sparse_k<NB, vdk::kEuclid, 1>(ksel, dedup, g, b, st, pdl, a);
    }
  }
  switch (key) {
    case 2: return launch_sparse_k<NB, vdk::kManhattan, 2>(ksel, dedup, g, b, st, pdl, a);
    case 0: return launch_sparse_k<NB, vdk::kManhattan, 0>(ksel, dedup, g, b, st, pdl, a);
    default: return launch_sparse_k<NB, vdk::kManhattan, 1>(ksel, dedup, g, b, st, pdl, a);
  }
}

int launch_pass_sparse(const vdk::PassArgs& a, dim3 grid, dim3 block, int32_t nb, int32_t metric, int key, int ksel,
                       bool dedup, cudaStream_t st, bool pdl) {
  const cudaError_t e = nb == VD_NB_MOORE
                            ? launch_sparse_nb<vdk::kMoore>(metric, key, ksel, dedup, grid, block, st, pdl, a)
                            : launch_sparse_nb<vdk::kVonNeumann>(metric, key, ksel, dedup, grid, block, st, pdl, a);
  if (e != cudaSuccess) return vd_cuda_check(e, "sparse jump pass launch");
  return vd_cuda_check(cudaGetLastError(), "sparse jump pass launch");
}

}  // namespace vdi
