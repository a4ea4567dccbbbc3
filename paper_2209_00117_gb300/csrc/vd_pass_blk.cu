// vd_pass_blk.cu -- the jump pass of the byte-offset key forms for steps
// k = 4, 8, 12, ... (k % 4 == 0), register-blocked over 2 x 2 quads.
//
// One jump pass (Table I for Moore, Section V-B for Von Neumann) gives pixel q
// the nearest of the seeds named at q and at q + o k.  With k a multiple of
// 4, pixel i of a 4-pixel quad takes exactly element i of each neighbouring
// 4-label vector, so a thread of the plain pass loads 9 (Moore) or 5 (Von
// Neumann) vectors and gathers a table entry for each label.  Here one
// thread owns the four quads at (x0 + a k, y + b k), a, b in {0, 1}: their
// neighbourhoods overlap, and the 16 (Moore) or 12 (Von Neumann) vectors at
// (x0 + c k, y + r k), c, r in {-1, 0, 1, 2}, serve all four -- each vector
// is loaded and its labels gathered once instead of up to four times.  The
// candidates each pixel scores, and so every result, are exactly those of
// the plain pass; the byte-offset key arithmetic and the winner check are the
// ones described at vdk::Quad8 (a quad that fails the check is recomputed by
// the clamped form, vdk::byte_fallback).
#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace vdk {

constexpr int kBlkThreadsX = 32;
constexpr int kBlkThreadsY = 4;

// Key of a candidate whose packed position is e, for the pixel whose bias
// word is kp = 2^15 - (x | y << 16) (Quad8): d = dx^2 + dy^2 from one dp4a,
// then (d, label) packed.  LB = 16: one byte permute puts d in the high half
// (PRMT) or a multiply-add does (mul = 2^16); LB > 16: d << LB plus the label
// (the wide form, a compile-time shift); LB = 0: d * mul + label with the
// runtime mul = 2^lb.
template <int LB, bool PRMT>
__device__ __forceinline__ uint32_t byte_key(uint32_t e, uint32_t kp, int c, uint32_t mul) {
  const uint32_t v = e + kp;
  const int d = __dp4a(static_cast<int>(v), static_cast<int>(v & 0x00FF00FFu), 0);
  if (LB == 16 && PRMT) return __byte_perm(static_cast<uint32_t>(c), static_cast<uint32_t>(d), 0x5410);
  if (LB > 16) return (static_cast<uint32_t>(d) << LB) + static_cast<uint32_t>(c);
  return static_cast<uint32_t>(d) * mul + static_cast<uint32_t>(c);
}

template <int NB>
__device__ __forceinline__ constexpr bool blk_uses(int c, int r, int qa, int qb) {
  // vector (c, r) is a candidate vector of quad (qa, qb)
  return NB == kMoore ? (c - qa >= -1 && c - qa <= 1 && r - qb >= -1 && r - qb <= 1)
                      : ((c == qa && r - qb >= -1 && r - qb <= 1) || (r == qb && c - qa >= -1 && c - qa <= 1));
}

// Folds vector (C, R) into every quad of the block that has it as a
// candidate vector (skipping quads outside the map).
template <int NB, int C, int R, int LB, bool PRMT, bool DEDUP>
__device__ __forceinline__ void blk_vector(const PassArgs& a, const int32_t* __restrict__ src, int x0, int y,
                                           const uint32_t (&kp)[2][2], const bool (&qv)[2][2],
                                           uint32_t (&best)[2][2][4]) {
  constexpr bool u00 = blk_uses<NB>(C, R, 0, 0), u10 = blk_uses<NB>(C, R, 1, 0);
  constexpr bool u01 = blk_uses<NB>(C, R, 0, 1), u11 = blk_uses<NB>(C, R, 1, 1);
  if (!(u00 || u10 || u01 || u11)) return;
  const int xs = x0 + C * a.k;
  const int ys = y + R * a.k;
  if (xs < 0 || xs >= a.pitch || ys < 0 || ys >= a.h) return;  // out of the map: not a candidate
  const int4 L = __ldg(reinterpret_cast<const int4*>(src + static_cast<int64_t>(ys) * a.pitch + xs));
  uint32_t p0, p1, p2, p3;
  p0 = __ldg(&a.ptable[L.x]);
  if (DEDUP) {
    p1 = p0;
    if (L.y != L.x) p1 = __ldg(&a.ptable[L.y]);
    p2 = p1;
    if (L.z != L.y) p2 = __ldg(&a.ptable[L.z]);
    p3 = p2;
    if (L.w != L.z) p3 = __ldg(&a.ptable[L.w]);
  } else {
    p1 = __ldg(&a.ptable[L.y]);
    p2 = __ldg(&a.ptable[L.z]);
    p3 = __ldg(&a.ptable[L.w]);
  }
  const uint32_t mul = a.bmul;
#define VD_BLK_FOLD(QA, QB)                                                                              \
  if ((QA == 0 && QB == 0) || qv[QA][QB]) {                                                             \
    best[QA][QB][0] = min(best[QA][QB][0], byte_key<LB, PRMT>(p0, kp[QA][QB], L.x, mul));              \
    best[QA][QB][1] = min(best[QA][QB][1], byte_key<LB, PRMT>(p1, kp[QA][QB] - 1u, L.y, mul));         \
    best[QA][QB][2] = min(best[QA][QB][2], byte_key<LB, PRMT>(p2, kp[QA][QB] - 2u, L.z, mul));         \
    best[QA][QB][3] = min(best[QA][QB][3], byte_key<LB, PRMT>(p3, kp[QA][QB] - 3u, L.w, mul));         \
  }
  if (u00) VD_BLK_FOLD(0, 0)
  if (u10) VD_BLK_FOLD(1, 0)
  if (u01) VD_BLK_FOLD(0, 1)
  if (u11) VD_BLK_FOLD(1, 1)
#undef VD_BLK_FOLD
}

// The winner check of the byte-offset form for one quad, then its store (or
// its recomputation by the clamped form).
template <int NB, bool WIDE, bool DEDUP>
__device__ __forceinline__ void blk_finish(const PassArgs& a, int x0, int y, const uint32_t (&b)[4]) {
  const uint32_t* __restrict__ arena = a.ptable - 1;
  constexpr uint32_t h = kByteWindow;
  const uint32_t mask = WIDE ? a.bmul - 1u : 0xFFFFu;
  const uint32_t wmask = WIDE ? a.bwin_mask : (0xFFFFu & ~(2u * h - 1u)) * 0x10001u;
  const uint32_t kw = (WIDE ? a.bwin_bias : h * 0x10001u) -
                      (static_cast<uint32_t>(x0) + (static_cast<uint32_t>(y) << 16));
  uint32_t bad = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t j = (b[i] + 1u) & mask;
    bad |= (__ldg(&arena[j]) + kw - static_cast<uint32_t>(i)) & wmask;
  }
  const uint32_t top = max(max(b[0], b[1]), max(b[2], b[3]));
  if (bad != 0 || top >= (WIDE ? a.blim : (h * h) << 16)) {
    byte_fallback<NB, 0, false, DEDUP>(a, x0, y);
    return;
  }
  store_quad(a, x0, y, static_cast<int>(b[0] & mask), static_cast<int>(b[1] & mask), static_cast<int>(b[2] & mask),
             static_cast<int>(b[3] & mask));
}

// Thread (t, u) owns the quads at (x0 + a k, y + b k): with q = k / 4 quads
// per k pixels, t = s q + i gives x0 = 2 k s + 4 i and u = s' k + j gives
// y = 2 k s' + j, so the threads of a warp (consecutive t) read consecutive
// 16-byte vectors within each k-wide run.
// MINB: resident blocks per SM the register budget is cut for (6: 80
// registers a thread, 8: 64).
template <int NB, bool WIDE, int LB, bool PRMT, bool DEDUP, int MINB>
__global__ void __launch_bounds__(kBlkThreadsX* kBlkThreadsY, MINB) k_pass_blk(PassArgs a) {
  pdl_trigger();
  pdl_wait();
  const int k = a.k;
  const int q = k >> 2;
  const int t = static_cast<int>(blockIdx.x) * kBlkThreadsX + static_cast<int>(threadIdx.x);
  const int u = static_cast<int>(blockIdx.y) * kBlkThreadsY + static_cast<int>(threadIdx.y);
  const int s = t / q, s2 = u / k;
  const int x0 = 2 * k * s + 4 * (t - s * q);
  const int y = 2 * k * s2 + (u - s2 * k);
  if (x0 >= a.pitch || y >= a.h) return;
  bool qv[2][2];
  qv[0][0] = true;
  qv[1][0] = x0 + k < a.pitch;
  qv[0][1] = y + k < a.h;
  qv[1][1] = qv[1][0] && qv[0][1];
  uint32_t kp[2][2];
#pragma unroll
  for (int qa = 0; qa < 2; ++qa)
#pragma unroll
    for (int qb = 0; qb < 2; ++qb)
      kp[qa][qb] = 0x8000u - (static_cast<uint32_t>(x0 + qa * k) + (static_cast<uint32_t>(y + qb * k) << 16));
  uint32_t best[2][2][4];
#pragma unroll
  for (int qa = 0; qa < 2; ++qa)
#pragma unroll
    for (int qb = 0; qb < 2; ++qb)
#pragma unroll
      for (int i = 0; i < 4; ++i) best[qa][qb][i] = 0xFFFFFFFFu;
  const int32_t* __restrict__ src = a.src;
#define VD_BLK_V(C, R)                                                      \
  blk_vector<NB, C, R, LB, PRMT, DEDUP>(a, src, x0, y, kp, qv, best); \
  group_fence();
  VD_BLK_V(-1, -1)
  VD_BLK_V(0, -1)
  VD_BLK_V(1, -1)
  VD_BLK_V(2, -1)
  VD_BLK_V(-1, 0)
  VD_BLK_V(0, 0)
  VD_BLK_V(1, 0)
  VD_BLK_V(2, 0)
  VD_BLK_V(-1, 1)
  VD_BLK_V(0, 1)
  VD_BLK_V(1, 1)
  VD_BLK_V(2, 1)
  VD_BLK_V(-1, 2)
  VD_BLK_V(0, 2)
  VD_BLK_V(1, 2)
  VD_BLK_V(2, 2)
#undef VD_BLK_V
  blk_finish<NB, WIDE, DEDUP>(a, x0, y, best[0][0]);
  if (qv[1][0]) blk_finish<NB, WIDE, DEDUP>(a, x0 + k, y, best[1][0]);
  if (qv[0][1]) blk_finish<NB, WIDE, DEDUP>(a, x0, y + k, best[0][1]);
  if (qv[1][1]) blk_finish<NB, WIDE, DEDUP>(a, x0 + k, y + k, best[1][1]);
}

}  // namespace vdk

namespace vdi {

template <int NB, bool WIDE, int LB, bool PRMT>
static cudaError_t launch_blk_t(bool dedup, int minb, dim3 g, dim3 b, cudaStream_t st, bool pdl,
                                const vdk::PassArgs& a) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  if (minb == 6) {
    if (dedup) return cudaLaunchKernelEx(&cfg, vdk::k_pass_blk<NB, WIDE, LB, PRMT, true, 6>, a);
    return cudaLaunchKernelEx(&cfg, vdk::k_pass_blk<NB, WIDE, LB, PRMT, false, 6>, a);
  }
  if (dedup) return cudaLaunchKernelEx(&cfg, vdk::k_pass_blk<NB, WIDE, LB, PRMT, true, 8>, a);
  return cudaLaunchKernelEx(&cfg, vdk::k_pass_blk<NB, WIDE, LB, PRMT, false, 8>, a);
}

template <int NB>
static cudaError_t launch_blk_nb(bool wide, int lb, int pack, bool dedup, int minb, dim3 g, dim3 b, cudaStream_t st,
                                 bool pdl, const vdk::PassArgs& a) {
  if (!wide) {
    return pack == 1 ? launch_blk_t<NB, false, 16, true>(dedup, minb, g, b, st, pdl, a)
                     : launch_blk_t<NB, false, 16, false>(dedup, minb, g, b, st, pdl, a);
  }
  if (pack == 2) {
    switch (lb) {
      case 17: return launch_blk_t<NB, true, 17, false>(dedup, minb, g, b, st, pdl, a);
      case 18: return launch_blk_t<NB, true, 18, false>(dedup, minb, g, b, st, pdl, a);
      case 19: return launch_blk_t<NB, true, 19, false>(dedup, minb, g, b, st, pdl, a);
      default: break;
    }
  }
  return launch_blk_t<NB, true, 0, false>(dedup, minb, g, b, st, pdl, a);
}

bool blk_applies(int32_t k, int key) { return k >= 4 && k % 4 == 0 && (key == 3 || key == 4); }

int launch_pass_blk(const vdk::PassArgs& a, int32_t nb, int key, bool dedup, int pack, int minb, cudaStream_t st,
                    bool pdl) {
  const int k = a.k;
  const int q = k / 4;
  const int64_t tcols = ((static_cast<int64_t>(a.pitch) + 2 * k - 1) / (2 * k)) * q;
  const int64_t trows = ((static_cast<int64_t>(a.h) + 2 * k - 1) / (2 * k)) * k;
  dim3 block(vdk::kBlkThreadsX, vdk::kBlkThreadsY);
  dim3 grid(static_cast<unsigned>((tcols + vdk::kBlkThreadsX - 1) / vdk::kBlkThreadsX),
            static_cast<unsigned>((trows + vdk::kBlkThreadsY - 1) / vdk::kBlkThreadsY));
  int lb = 16;
  byte_key_window(a.n_seeds, &lb);
  const bool wide = key == 4;
  const cudaError_t e = nb == VD_NB_MOORE
                            ? launch_blk_nb<vdk::kMoore>(wide, lb, pack, dedup, minb, grid, block, st, pdl, a)
                            : launch_blk_nb<vdk::kVonNeumann>(wide, lb, pack, dedup, minb, grid, block, st, pdl, a);
  if (e != cudaSuccess) return vd_cuda_check(e, "blocked jump pass launch");
  return vd_cuda_check(cudaGetLastError(), "blocked jump pass launch");
}

}  // namespace vdi
