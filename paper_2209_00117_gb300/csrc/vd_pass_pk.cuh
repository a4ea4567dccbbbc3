// vd_pass_pk.cuh -- dJFA passes over a position-tagged label map.
//
// A pass (Table I for Moore, Section V-B for Von Neumann) scores, for every
// pixel, the seeds named at it and at its neighbours k away.  The plain pass
// reads each candidate's position from the seed table: one dependent gather
// per candidate, and with it the address arithmetic and, de-duplicated, a
// compare and a move.  Inside a dJFA frame (Eq. 4's schedule after the stamp)
// the maps between the first and the last pass are never seen outside the
// frame, so there each 32-bit word carries, beside the label, the low M bits
// of its seed's x and y, and a candidate is scored from the word alone:
//
//   M = 6, 7 ("wide"): bits [0, 24 - M) label, [24 - M, 24) x mod 2^M,
//                      bit 24 set (guard), [32 - M, 32) y mod 2^M; with
//                      M = 6 bit 25 marks an empty pixel.
//   M = 8 ("narrow"):  bits [0, 8) label bits 0-7, [8, 16) x mod 256,
//                      [16, 23) label bits 8-14, bit 23 set (guard),
//                      [24, 32) y mod 256.
//   M = 4 ("split"):   bits [0, 20) label bits 0-19, [20, 24) x mod 16,
//                      [24, 26) label bits 20-21, bit 26 set (guard),
//                      bit 27 marks an empty pixel, [28, 32) y mod 16
//                      (up to 2^22 seeds).
//
// For a pixel whose own fields P sit in the same places, v = w - P holds
// (x - x_p) mod 2^M and (y - y_p) mod 2^M at the top of their bytes: the guard
// bit absorbs the borrow out of the x field, so the y field is exact, and the
// label bits below the x field see no borrow at all.  Masked to the fields,
// the two bytes read as signed numbers are 2^(8-M) dx and 2^(8-M) dy for every
// seed with dx, dy in [-2^(M-1), 2^(M-1)) (the window), and one dp4a gives
// 4^(8-M) (dx^2 + dy^2).  The key is d * 2^(24-M) + label (wide: the label
// masked out of the word and one multiply-add) or d * 2^16 + 2^15 + label
// (narrow: one byte permute of the word and d).  Per candidate: a subtraction,
// a mask, the dp4a, the key pack (wide: and the label mask) and a minimum; no
// gather.  No key wraps: wide keys lie below 2^31, narrow ones hold d <= 2^15
// in their upper 16 bits (keys compare as unsigned).  The split layout's
// label code (its label bits where the word holds them, an order-preserving
// image of the label) spans 26 bits, which leaves 6 bits for d: its key is
// min(d, 63) * 2^26 + code, one more minimum a candidate, and the winner
// check accepts d < 63 only (a saturated key carries no distance).
//
// Outside the window the fields alias and a key may be anything, and the
// byte-offset pass's winner check applies unchanged: each pixel's winner is
// looked up in the position table, and when it lies inside the window at
// d < h^2 (h = 2^(M-1)) every seed outside the window lies at least h^2 away
// and every seed inside was scored exactly, so the winner is the exact one
// (the lowest label among the nearest, the key's low bits being the label).
// Otherwise the quad is recomputed exactly from the words' labels with the
// 64-bit (distance, label) key.  The label code 2^lb - 1 -- the empty code,
// and with M = 6 and 2^18 seeds also the last seed -- indexes the far entry
// of the position table and so always takes the recomputation.
//
// A frame runs its first packed pass on the plain map (the byte-offset fold
// with gathers; for the split layout, whose labels leave the byte-offset key
// too narrow a window, the clamped 32-bit fold) writing words, the passes
// after it word to word, and its last pass writes plain labels again.
#pragma once

#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace vdk {

template <int M>
struct Pk {
  static constexpr bool kNarrow = M == 8;
  static constexpr bool kSplit = M == 4;
  static constexpr int kLb = kNarrow ? 15 : kSplit ? 26 : 24 - M;  // label code bits
  static constexpr int kKs = kNarrow ? 16 : kLb;                    // key = d * 2^kKs + ...
  // label code mask; all ones: empty
  static constexpr uint32_t kLm = kSplit ? 0x030FFFFFu : (1u << kLb) - 1u;
  static constexpr uint32_t kH = 1u << (M - 1);  // window: dx, dy in [-kH, kH)
  static constexpr uint32_t kXm = (1u << M) - 1u;
  static constexpr int kXs = kNarrow ? 8 : kSplit ? 20 : kLb;  // x field shift
  static constexpr int kYs = 32 - M;                           // y field shift
  static constexpr uint32_t kFm = (kXm << kXs) | (kXm << kYs);
  static constexpr uint32_t kG = kNarrow ? 0x00800000u : kSplit ? 0x04000000u : 0x01000000u;
  // empty flag (M = 6 and 4, whose all-ones code is also the last seed's)
  static constexpr uint32_t kEf = M == 6 ? 0x02000000u : kSplit ? 0x08000000u : 0u;
  static constexpr uint32_t kEmpty = kNarrow ? (0xFFu | (0x7Fu << 16) | kG) : (kLm | kG | kEf);
  // keys at or above this fail the winner check: d >= h^2 (split: d >= 63,
  // the saturated keys)
  static constexpr uint32_t kLim = kSplit ? 63u << kKs : (kH * kH) << kKs;
  // the dp4a sum of the split layout is 256 d, saturated at 256 * 63
  static constexpr uint32_t kSat = 63u * 256u;

  // The fields of pixel (x, y), negated: v = w + neg_pix(x, y).
  __device__ __forceinline__ static uint32_t neg_pix(uint32_t x, uint32_t y) {
    return 0u - (((x & kXm) << kXs) | ((y & kXm) << kYs));
  }
  // The label a code (of a word or a key) names (split: its bits joined).
  __device__ __forceinline__ static uint32_t code_label(uint32_t c) {
    return kSplit ? ((c & 0xFFFFFu) | ((c >> 4) & 0x300000u)) : (c & kLm);
  }
  // The label a word names, -1 for the empty word.
  __device__ __forceinline__ static int label(uint32_t w) {
    if (kEf) return (w & kEf) ? -1 : static_cast<int>(code_label(w));
    const uint32_t c = kNarrow ? ((w & 0xFFu) | ((w >> 8) & 0x7F00u)) : (w & kLm);
    return c == kLm ? -1 : static_cast<int>(c);
  }
  // The label bits of label l where a word holds them.
  __device__ __forceinline__ static uint32_t code(uint32_t l) {
    return kSplit ? (l & 0xFFFFFu) | ((l & 0x300000u) << 4) : l;
  }
  // The word of label l >= 0 whose seed lies at e = x | y << 16.
  __device__ __forceinline__ static uint32_t word(uint32_t l, uint32_t e) {
    if (kNarrow) return (l & 0xFFu) | ((e & 0xFFu) << 8) | ((l & 0x7F00u) << 8) | kG | ((e >> 16) << 24);
    return code(l) | kG | ((e & kXm) << kXs) | (((e >> 16) & kXm) << kYs);
  }
  // Key of word w for the pixel with negated fields pn.
  __device__ __forceinline__ static uint32_t key(uint32_t w, uint32_t pn) {
    const uint32_t b = (w + pn) & kFm;
    const uint32_t d = static_cast<uint32_t>(__dp4a(static_cast<int>(b), static_cast<int>(b), 0));
    if (kNarrow) return __byte_perm(w, d, 0x5420);
    if (kSplit) return min(d, kSat) * (1u << 18) + (w & kLm);
    return d * (1u << (8 + M)) + (w & kLm);
  }
  // The position-table index of a key's label (far entry first): (label + 1)
  // modulo the code's range, so that the empty code lands on the far entry.
  __device__ __forceinline__ static uint32_t index(uint32_t key) {
    if (kSplit) return (code_label(key) + 1u) & 0x3FFFFFu;
    return (key + 1u) & kLm;
  }
  // The winner's word from its key and its seed position e (check passed).
  __device__ __forceinline__ static uint32_t word_of_key(uint32_t key, uint32_t e) {
    if (kNarrow) return __byte_perm(key, e, 0x6140);
    return (key & kLm) | fields(e);
  }
  // A word's bits but the label, for the seed at e (wide layouts).
  __device__ __forceinline__ static uint32_t fields(uint32_t e) {
    return kG | ((e << kXs) & (kXm << kXs)) | ((e << (16 - M)) & (kXm << kYs));
  }
};

__device__ __forceinline__ uint4 words4(const int32_t* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
__device__ __forceinline__ uint32_t words1(const int32_t* p) {
  return static_cast<uint32_t>(__ldg(p));
}
__device__ __forceinline__ uint2 words2(const int32_t* p) { return __ldg(reinterpret_cast<const uint2*>(p)); }

// The exact recomputation of one quad (x0 .. x0 + 3, y): for each pixel the
// least (distance^2, label) over its candidates (Table I / Section V-B),
// candidates outside the map and empty ones skipped, read from a plain map
// (PKIN false) or a packed one; written plain or packed (PKOUT).  Per pixel
// all candidate words are loaded at once, then all their seed positions, so
// that a quad costs two memory round trips a pixel rather than two a
// candidate: with 2^18 seeds on 8192^2 about 1.5% of the first pass's quads
// land here (a seed beyond the +-32 window of a k = 32 neighbour aliasing
// to a short offset), enough warps that a serial recomputation held their
// blocks and dominated that pass.  Out of line (with the border blocks'
// path also out of line, measured 6% faster a dJFA frame than either inline
// on the GB300).
template <int NB, int M, bool PKIN, bool PKOUT>
__device__ __noinline__ void pk_exact_quad(const PassArgs a, int x0, int y) {
  using F = Pk<M>;
  constexpr int kN = NB == kMoore ? 9 : 5;
  // candidate offsets in units of k: the pixel, its four axis neighbours,
  // then (Moore) the four diagonal ones
  constexpr int kOx[9] = {0, -1, 1, 0, 0, -1, 1, -1, 1};
  constexpr int kOy[9] = {0, 0, 0, -1, 1, -1, -1, 1, 1};
  uint32_t out[4];
#pragma unroll 1
  for (int i = 0; i < 4; ++i) {
    const int x = x0 + i;
    if (x >= a.w) {
      out[i] = PKOUT ? F::kEmpty : 0xFFFFFFFFu;
      continue;
    }
    int lab[kN];
#pragma unroll
    for (int c = 0; c < kN; ++c) {
      const int qx = x + kOx[c] * a.k, qy = y + kOy[c] * a.k;
      const bool in = qx >= 0 && qx < a.w && qy >= 0 && qy < a.h;
      const uint32_t wv = in ? static_cast<uint32_t>(__ldg(a.src + static_cast<int64_t>(qy) * a.pitch + qx))
                             : 0xFFFFFFFFu;
      lab[c] = !in ? -1 : PKIN ? F::label(wv) : static_cast<int>(wv);
    }
    uint32_t e[kN];
#pragma unroll
    for (int c = 0; c < kN; ++c) e[c] = lab[c] >= 0 ? __ldg(&a.ptable[lab[c]]) : 0u;
    unsigned long long best = ~0ull;
    uint32_t eb = 0;
#pragma unroll
    for (int c = 0; c < kN; ++c) {
      if (lab[c] < 0) continue;
      const int sx = static_cast<int>(e[c] & 0xFFFFu) - x;
      const int sy = static_cast<int>(e[c] >> 16) - y;
      const uint32_t d = static_cast<uint32_t>(sx * sx) + static_cast<uint32_t>(sy * sy);
      const unsigned long long kk = (static_cast<unsigned long long>(d) << 32) | static_cast<uint32_t>(lab[c]);
      if (kk < best) {
        best = kk;
        eb = e[c];
      }
    }
    const int l = best == ~0ull ? -1 : static_cast<int>(static_cast<uint32_t>(best));
    if (PKOUT) out[i] = l < 0 ? F::kEmpty : F::word(static_cast<uint32_t>(l), eb);
    else out[i] = static_cast<uint32_t>(l);
  }
  *reinterpret_cast<uint4*>(a.dst + static_cast<int64_t>(y) * a.pitch + x0) = make_uint4(out[0], out[1], out[2], out[3]);
}

// The winner check and the store of one quad whose keys are d * 2^ks + code
// (code = label, its low lb bits; all ones: empty): e = the position-table
// entry at (code + 1) mod 2^lb (split layout: (label + 1) mod 2^22) with the
// far position first, in the window
// [-h, h) around each pixel, and every d < h^2.  lm = 2^lb - 1; the window
// kw = h * 0x10001 - (x0 | y << 16), wmask = (0xFFFF & ~(2h - 1)) * 0x10001,
// lim = h^2 << ks.  PKOUT: words of layout M from the keys (key form KF: 0
// the plain byte-offset key, labels in the low lb bits; 1 this layout's;
// 2 either, labels in the low lb bits, with each seed's word bits of a wide
// layout read from a.pkf beside its position, as the frame's stamp wrote
// them).  Returns false when the quad must be recomputed.
template <int M, int KF, bool PKOUT, bool IN>
__device__ __forceinline__ bool pk_check_store(const PassArgs& a, const uint32_t (&b)[4], int x0, int y,
                                               uint32_t lm, uint32_t kw, uint32_t wmask, uint32_t lim) {
  using F = Pk<M>;
  const uint32_t* __restrict__ arena = a.ptable - 1;
  uint32_t e[4], f[4];
  uint32_t bad = 0, top = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // (the split layout's code is not the label: its index joins the bits)
    const uint32_t j = F::kSplit ? F::index(b[i]) : (b[i] + 1u) & lm;
    if (KF == 2) {
      const uint2 ef = __ldg(&a.pkf[j]);
      e[i] = ef.x;
      f[i] = ef.y;
    } else {
      e[i] = __ldg(&arena[j]);
    }
    // (dx + h) | (dy + h) << 16 has no bit at or above 2h in either half
    // exactly when dx, dy lie in [-h, h)
    const uint32_t t = (e[i] + kw - static_cast<uint32_t>(i)) & wmask;
    if (IN || x0 + i < a.w) {
      bad |= t;
      top = max(top, b[i]);
    }
  }
  if (bad != 0 || top >= lim) return false;
  uint32_t o[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // (the plain narrow key's label bytes are bytes 0 and 1, the second
    // below 0x80: one byte permute and the guard bit)
    if (PKOUT)
      o[i] = KF == 2   ? (b[i] & lm) | f[i]
             : KF == 1 ? F::word_of_key(b[i], e[i])
             : M == 8  ? __byte_perm(b[i], e[i], 0x6140) | F::kG
                       : F::word(b[i] & lm, e[i]);
    else o[i] = F::kSplit ? F::code_label(b[i]) : b[i] & lm;
    if (!IN && x0 + i >= a.w) o[i] = PKOUT ? F::kEmpty : 0xFFFFFFFFu;
  }
  *reinterpret_cast<uint4*>(a.dst + static_cast<int64_t>(y) * a.pitch + x0) = make_uint4(o[0], o[1], o[2], o[3]);
  return true;
}

// The first packed pass of a frame: the byte-offset fold on the plain map
// (as the plain pass), its winner check, then words of layout M.
template <int NB, int KSEL, int M, bool DEDUP, bool IN>
__device__ __forceinline__ void pk_first_quad(const PassArgs& a, int x0, int y) {
  constexpr bool kWide = M != 8;
  Quad8<false, DEDUP, !kWide && KSEL != 0> q(a, x0, y);
  fold_all<NB, KSEL, false, IN>(q, a, x0, y);
  constexpr uint32_t h = kByteWindow;
  const uint32_t lm = kWide ? a.bmul - 1u : 0xFFFFu;
  const uint32_t wmask = kWide ? a.bwin_mask : (0xFFFFu & ~(2u * h - 1u)) * 0x10001u;
  const uint32_t kw = (kWide ? a.bwin_bias : h * 0x10001u) -
                      (static_cast<uint32_t>(x0) + (static_cast<uint32_t>(y) << 16));
  const uint32_t lim = kWide ? a.blim : (h * h) << 16;
  // words of a wide layout take their bits from a.pkf
  if (!pk_check_store<M, kWide ? 2 : 0, true, IN>(a, q.b, x0, y, lm, kw, wmask, lim))
    pk_exact_quad<NB, M, false, true>(a, x0, y);
}

// The split layout's first packed pass: the clamped 32-bit fold on the plain
// map (as the plain pass: exact while every pixel's best lies below the cap),
// then words from the labels and the seeds' word bits in a.pkf (which carry
// the labels' upper bits); a quad whose best reaches the cap is recomputed.
template <int NB, int KSEL, bool DEDUP, bool IN>
__device__ __forceinline__ void pk_first_quad32(const PassArgs& a, int x0, int y) {
  using F = Pk<4>;
  Quad32<false, DEDUP> q(a, x0, y);
  fold_all<NB, KSEL, false, IN>(q, a, x0, y);
  if (max(max(q.b[0], q.b[1]), max(q.b[2], q.b[3])) >= (a.cap - 1u) * a.mul) {
    pk_exact_quad<NB, 4, false, true>(a, x0, y);
    return;
  }
  const uint32_t mask = a.mul - 1u;
  uint32_t o[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t l = q.b[i] & mask;
    o[i] = (l & 0xFFFFFu) | __ldg(&a.pkf[l + 1u].y);
    if (!IN && x0 + i >= a.w) o[i] = F::kEmpty;
  }
  *reinterpret_cast<uint4*>(a.dst + static_cast<int64_t>(y) * a.pitch + x0) = make_uint4(o[0], o[1], o[2], o[3]);
}

// One packed pass (words in) for the quad (x0 .. x0 + 3, y).  Candidate order
// does not matter (the key is a total order).  Out-of-range side candidates
// take the same row's word at the pixel (scored anyway); out-of-range rows are
// skipped.
template <int NB, int KSEL, int M, bool PKOUT, bool IN>
__device__ __forceinline__ void pk_quad(const PassArgs& a, int x0, int y) {
  using F = Pk<M>;
  // element indices fit 32 bits (sides up to 32768): one base pointer and
  // 32-bit offsets keep the six runtime-step addresses cheap in registers
  const int k = a.k;
  const int32_t* __restrict__ src = a.src;
  const int c0 = y * a.pitch + x0;
  const int kp = k * a.pitch;
  const uint32_t pn = F::neg_pix(static_cast<uint32_t>(x0), static_cast<uint32_t>(y));
  // pixel i's fields: pn minus i in the x field (one three-input add with
  // the word, the offset an immediate)
#define pi(i) (pn - (static_cast<uint32_t>(i) << F::kXs))
  uint32_t b[4];
  const uint4 own = words4(src + c0);
  const bool up_ok = IN || y - k >= 0;
  const bool dn_ok = IN || y + k < a.h;
  const uint32_t ow[4] = {own.x, own.y, own.z, own.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) b[i] = F::key(ow[i], pi(i));
  // the side candidates of one row (index r of its element at x0), `mid` its
  // vector at x0
  auto sides = [&](int r, const uint32_t (&mid)[4]) {
    if (KSEL == 0) {
      const bool lok = IN || x0 - k >= 0, rok = IN || x0 + k < a.pitch;
      const uint4 L = lok ? words4(src + r - k) : make_uint4(mid[0], mid[1], mid[2], mid[3]);
      const uint32_t l[4] = {L.x, L.y, L.z, L.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = min(b[i], F::key(l[i], pi(i)));
      group_fence();
      const uint4 R = rok ? words4(src + r + k) : make_uint4(mid[0], mid[1], mid[2], mid[3]);
      const uint32_t rv[4] = {R.x, R.y, R.z, R.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) b[i] = min(b[i], F::key(rv[i], pi(i)));
    } else if (KSEL == 1) {
      // left of pixel i: column x0 + i - 1; right: x0 + i + 1
      const uint32_t wl = (IN || x0 >= 4) ? words1(src + r - 1) : mid[0];
      const uint32_t wr = (IN || x0 + 4 < a.pitch) ? words1(src + r + 4) : mid[3];
      b[0] = min(b[0], min(F::key(wl, pi(0)), F::key(mid[1], pi(0))));
      b[1] = min(b[1], min(F::key(mid[0], pi(1)), F::key(mid[2], pi(1))));
      b[2] = min(b[2], min(F::key(mid[1], pi(2)), F::key(mid[3], pi(2))));
      b[3] = min(b[3], min(F::key(mid[2], pi(3)), F::key(wr, pi(3))));
    } else {
      // left of pixel i: column x0 + i - 2; right: x0 + i + 2
      const uint2 wl = (IN || x0 >= 4) ? words2(src + r - 2) : make_uint2(mid[0], mid[1]);
      const uint2 wr = (IN || x0 + 4 < a.pitch) ? words2(src + r + 4) : make_uint2(mid[2], mid[3]);
      b[0] = min(b[0], min(F::key(wl.x, pi(0)), F::key(mid[2], pi(0))));
      b[1] = min(b[1], min(F::key(wl.y, pi(1)), F::key(mid[3], pi(1))));
      b[2] = min(b[2], min(F::key(mid[0], pi(2)), F::key(wr.x, pi(2))));
      b[3] = min(b[3], min(F::key(mid[1], pi(3)), F::key(wr.y, pi(3))));
    }
  };
  // the row's own vector at x0 (the vertical candidates), then its sides
  auto row_all = [&](int r) {
    const uint4 V = words4(src + r);
    const uint32_t v[4] = {V.x, V.y, V.z, V.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) b[i] = min(b[i], F::key(v[i], pi(i)));
    if (NB == kMoore) sides(r, v);
  };
  // one row's loads in flight at a time (group_fence): the register budget
  // of the launch shape holds no more
  sides(c0, ow);
  group_fence();
  if (up_ok) row_all(c0 - kp);
  group_fence();
  if (dn_ok) row_all(c0 + kp);
  const uint32_t kw = F::kH * 0x10001u - (static_cast<uint32_t>(x0) + (static_cast<uint32_t>(y) << 16));
  const uint32_t wmask = (0xFFFFu & ~(2u * F::kH - 1u)) * 0x10001u;
  // words out of a wide layout take their bits from a.pkf
  constexpr int kf = PKOUT && M != 8 ? 2 : 1;
  if (!pk_check_store<M, kf, PKOUT, IN>(a, b, x0, y, F::kLm, kw, wmask, F::kLim))
    pk_exact_quad<NB, M, true, PKOUT>(a, x0, y);
#undef pi
}

// The blocks within k of the map border (a few percent of them) run out of
// line, so that the interior path keeps a register allocation of its own.
template <int NB, int KSEL, int M, int MODE, bool DEDUP>
__device__ __noinline__ void pk_edge_quad(const PassArgs a, int x0, int y) {
  if (MODE == 0 && M == 4) pk_first_quad32<NB, KSEL, DEDUP, false>(a, x0, y);
  else if (MODE == 0) pk_first_quad<NB, KSEL, M, DEDUP, false>(a, x0, y);
  else pk_quad<NB, KSEL, M, MODE == 1, false>(a, x0, y);
}

#ifndef VD_PK_MIN_BLOCKS
#define VD_PK_MIN_BLOCKS 16
#endif

// The row order of k_pass (row-blocks in k-strided bands when band_m > 1) and
// its block-uniform interior test, in blocks of vdi::pk_threads threads (256
// for the Von Neumann passes on words, 128 otherwise; 32 registers a thread,
// the split layout's first pass the clamped plain pass's 48).
// MODE 0: plain map in, words out (DEDUP: the fold's gathers de-duplicated);
// 1: words in and out; 2: words in, plain labels out.
template <int NB, int KSEL, int M, int MODE, bool DEDUP = false>
__global__ void __launch_bounds__(vdi::pk_threads(NB, MODE),
                                  (MODE == 0 && M == 4 ? VD_PASS_MIN_BLOCKS : VD_PK_MIN_BLOCKS) * 128 /
                                      vdi::pk_threads(NB, MODE))
    k_pass_pk(PassArgs a) {
  pdl_trigger();
  pdl_wait();
  const int x0 = 4 * static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
  int rb = blockIdx.y;
  if (a.band_m > 1) rb = (blockIdx.y % a.band_t) * a.band_m + blockIdx.y / a.band_t;
  const int yb = rb * static_cast<int>(blockDim.y);
  const int y = yb + static_cast<int>(threadIdx.y);
  if (x0 >= a.pitch || y >= a.h) return;
  const int xb = 4 * static_cast<int>(blockIdx.x * blockDim.x);
  const bool in = xb - a.k >= 0 && xb + 4 * static_cast<int>(blockDim.x) + a.k <= a.w && yb - a.k >= 0 &&
                  yb + static_cast<int>(blockDim.y) + a.k <= a.h;
  if (!in) pk_edge_quad<NB, KSEL, M, MODE, DEDUP>(a, x0, y);
  else if (MODE == 0 && M == 4) pk_first_quad32<NB, KSEL, DEDUP, true>(a, x0, y);
  else if (MODE == 0) pk_first_quad<NB, KSEL, M, DEDUP, true>(a, x0, y);
  else pk_quad<NB, KSEL, M, MODE == 1, true>(a, x0, y);
}

}  // namespace vdk

namespace vdi {

using PkKernel = void (*)(vdk::PassArgs);

template <int NB, int KSEL, int M>
static PkKernel pk_kernel(int mode, bool dedup) {
  if (mode == 0) return dedup ? vdk::k_pass_pk<NB, KSEL, M, 0, true> : vdk::k_pass_pk<NB, KSEL, M, 0, false>;
  if (mode == 1) return vdk::k_pass_pk<NB, KSEL, M, 1>;
  return vdk::k_pass_pk<NB, KSEL, M, 2>;
}

template <int NB, int M>
static PkKernel pk_kernel_nb(int ksel, int mode, bool dedup) {
  if (ksel == 1) return pk_kernel<NB, 1, M>(mode, dedup);
  if (ksel == 2) return pk_kernel<NB, 2, M>(mode, dedup);
  return pk_kernel<NB, 0, M>(mode, dedup);
}

template <int M>
int launch_pass_pk_m(const vdk::PassArgs& a, dim3 grid, dim3 block, int32_t nb, int ksel, int mode,
                     bool dedup, cudaStream_t st, bool pdl) {
  const PkKernel fn = nb == VD_NB_MOORE ? pk_kernel_nb<vdk::kMoore, M>(ksel, mode, dedup)
                                        : pk_kernel_nb<vdk::kVonNeumann, M>(ksel, mode, dedup);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fn, a);
  if (e != cudaSuccess) return vd_cuda_check(e, "packed jump pass launch");
  return vd_cuda_check(cudaGetLastError(), "packed jump pass launch");
}

}  // namespace vdi
