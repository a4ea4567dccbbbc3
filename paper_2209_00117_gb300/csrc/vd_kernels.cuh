// vd_kernels.cuh -- sm_103a kernels of the jump-flooding hot path.
//
// Label maps are row-major int32 with a row pitch that is a multiple of 32
// elements (128 bytes); columns in [w, pitch) always hold -1, so a neighbour
// that falls into the padding reads as "empty" without a bounds test.  Seeds
// are int2 (x, y).  Every kernel here is a pure gather or a per-seed scatter:
// nothing waits on anything, so no launch can hang.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vdk {

constexpr int kEuclid = 0;
constexpr int kManhattan = 1;
constexpr int kMoore = 0;
constexpr int kVonNeumann = 1;

// Distance of Section II (squared Euclidean) or Section V-C (Manhattan),
// exact in 32 bits for grid sides up to 32768 (2 * 32767^2 < 2^31).
template <int METRIC>
__device__ __forceinline__ uint32_t seed_dist(int2 s, int x, int y) {
  const int dx = s.x - x;
  const int dy = s.y - y;
  if (METRIC == kManhattan) return static_cast<uint32_t>(abs(dx) + abs(dy));
  return static_cast<uint32_t>(dx * dx + dy * dy);
}

// Seed table entry used by the jump passes: {x | y << 16, x^2 + y^2}, 8 bytes
// (the passes are bound by the bytes that gathers return to registers, so
// the entry is kept as small as the key allows).  The table is stored with one
// sentinel entry in front, so entry -1 (the empty label) reads {0, INT32_MAX}:
// an empty candidate then loses every Euclidean comparison without a branch.
//
// Euclidean pass key for pixel q = (x, y) and seed s:
//   key = |s|^2 - 2 x s.x - 2 y s.y = d^2(s, q) - |q|^2,
// which orders the candidates of one pixel exactly as d^2 does (|q|^2 is the
// same for all of them), costs two multiply-adds and fits in int32.
// Manhattan key: |s.x - x| + |s.y - y|, with the empty label forced to a key
// above any real one.
constexpr int kSentinelNorm = 0x7FFFFFFF;

__device__ __forceinline__ int2 table_entry(int2 p) {
  return make_int2(p.x | (p.y << 16), p.x * p.x + p.y * p.y);
}

template <int METRIC>
__device__ __forceinline__ int table_key(int2 e, int c, int m2x, int m2y, int x, int y) {
  const int sx = e.x & 0xFFFF;
  const int sy = static_cast<int>(static_cast<unsigned int>(e.x) >> 16);
  if (METRIC == kManhattan) return c < 0 ? 0x40000000 : abs(sx - x) + abs(sy - y);
  // two's-complement wrap of the intermediate sums is harmless: the final
  // value is exact (|key| < 2^31)
  return static_cast<int>(static_cast<uint32_t>(e.y) + static_cast<uint32_t>(m2x) * static_cast<uint32_t>(sx) +
                          static_cast<uint32_t>(m2y) * static_cast<uint32_t>(sy));
}

// (key, label) packed into one int64: the signed high word orders by key, the
// low word (label as unsigned) breaks ties toward the lowest index, so the
// distance comparison of Section III with its lowest-index tie rule is one
// 64-bit minimum.  Label -1 only ever comes with the sentinel key.
__device__ __forceinline__ long long pack_key(int key, int c) {
  return (static_cast<long long>(key) << 32) | static_cast<unsigned int>(c);
}

template <int METRIC, bool COH = false>
__device__ __forceinline__ long long cand(int c, const int2* __restrict__ table, int m2x, int m2y, int x,
                                          int y) {
  const int2 e = COH ? __ldca(&table[c]) : __ldg(&table[c]);
  return pack_key(table_key<METRIC>(e, c, m2x, m2y, x, y), c);
}

// Folds candidate c into the packed best b.
template <int METRIC, bool COH = false>
__device__ __forceinline__ long long fold(long long b, int c, const int2* __restrict__ table, int m2x,
                                          int m2y, int x, int y) {
  return min(b, cand<METRIC, COH>(c, table, m2x, m2y, x, y));
}

// Kept for the kernels that read plain int2 positions (similarity, exact).
template <int METRIC>
__device__ __forceinline__ void consider(int c, const int2* __restrict__ seeds, uint32_t n, int x,
                                         int y, uint32_t& bd, int& bl) {
  if (static_cast<uint32_t>(c) < n && c != bl) {
    const uint32_t d = seed_dist<METRIC>(__ldg(&seeds[c]), x, y);
    if (d < bd || (d == bd && c < bl)) {
      bd = d;
      bl = c;
    }
  }
}

// Label-map and seed-table loads.  Separate launches use the read-only
// (non-coherent) path, ld.global.nc.  A persistent launch rewrites maps and
// tables between its grid barriers, and the read-only path is only defined
// for data that no thread writes during the launch, so it uses ordinary
// loads (ld.global.ca, cached in L1) instead: its grid barrier is a release
// (every thread's stores, the block barrier, then a gpu-scope fence and the
// atomic arrival) matched by an acquire (the spin read of the generation
// word, a gpu-scope fence, then the block barrier), so under the PTX memory
// model every load after the barrier observes every store made before it --
// an L1 line cached in an earlier round included.
template <bool COHERENT>
__device__ __forceinline__ int4 map4(const int32_t* p) {
  if (COHERENT) return __ldca(reinterpret_cast<const int4*>(p));
  return __ldg(reinterpret_cast<const int4*>(p));
}

template <bool COHERENT>
__device__ __forceinline__ int map1(const int32_t* p) {
  if (COHERENT) return __ldca(p);
  return __ldg(p);
}

template <bool COHERENT>
__device__ __forceinline__ int2 map2(const int32_t* p) {
  if (COHERENT) return __ldca(reinterpret_cast<const int2*>(p));
  return __ldg(reinterpret_cast<const int2*>(p));
}

struct PassArgs {
  const int32_t* __restrict__ src;
  int32_t* __restrict__ dst;
  const int2* __restrict__ table;       // {x | y << 16, x^2 + y^2}; entry -1 is the sentinel
  const uint32_t* __restrict__ ptable;  // positions x | y << 16; entry -1 is the far position
  uint32_t cap;                         // clamped-key passes: distance cap 2^(32 - lb) - 1
  uint32_t mul;                         // and 2^lb, lb = bits of the largest label
  uint32_t n_seeds;
  // byte-offset passes: bmul = 2^lb (2^16 below 2^16 seeds, a runtime value:
  // see Quad8::key); the wide form (2^16 seeds and more, 2^lb > n_seeds) also
  // reads its window h as bwin_bias = h * 0x10001, bwin_mask =
  // (0xFFFF & ~(2h - 1)) * 0x10001 and blim = h^2 * 2^lb
  uint32_t bmul, bwin_bias, bwin_mask, blim;
  int w, h, pitch, k;
  int band_m;  // > 1: visit row-blocks in k-strided bands (band_m = k / rows per block)
  int band_t;  // row-blocks per band residue class
  int y0, y_end;  // k_pass writes rows [y0, y_end) of dst (the whole map: 0, h)
  // position-tagged passes (wide layouts): n + 1 entries {x | y << 16, the
  // seed's word bits but the label}, [0] the far position; written by the
  // frame's stamp (k_stamp_min)
  const uint2* __restrict__ pkf;
};

// Stops the compiler from hoisting later loads above this point, which keeps
// only one neighbour group's gathers in flight per thread (the register
// budget of the pass launch shape) and leaves latency hiding to the many
// resident warps.
__device__ __forceinline__ void group_fence() { asm volatile("" ::: "memory"); }

// Programmatic dependent launch.  pdl_trigger lets the next kernel on the
// stream, when it was launched with programmatic stream serialization, be
// scheduled onto SMs this grid frees while it drains; pdl_wait blocks until
// the grid this one depends on has completed and its writes are visible.  A
// kernel of such a chain calls both before its first global-memory access.
// For a kernel launched without the attribute the wait returns at once (its
// predecessor has completed by stream order).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Packed position table of the 32-bit key forms: entry k + 1 holds seed k as
// x | y << 16 (both below 2^15); entry 0 (label -1) holds the far position
// (kFarX, 0).  From any pixel of a grid up to 32768 wide that position lies
// at squared distance [2^28, 49151^2 + 32767^2]: at or above every clamp cap
// (2^28 - 1 at most) and below 2^32.
constexpr uint32_t kFarX = 49151;

__host__ __device__ __forceinline__ uint32_t pack_pos(int x, int y) {
  return static_cast<uint32_t>(x) | (static_cast<uint32_t>(y) << 16);
}

// The four pixels (x0 .. x0+3, y) owned by one thread and their best
// candidate so far.  Each key form gathers a seed's table entry once per
// label and turns it into a "prepared position" (int2) holding what the four
// pixels of the row share -- the seed's x and its y-term -- so that a
// gathered entry can serve every pixel of the quad it is a candidate for.
//   pos(c)          gather + prepare label c (c = -1: the sentinel entry)
//   set(i, p, c)    best of pixel x0 + i := candidate (p, c)
//   fold(i, p, c)   best of pixel x0 + i := min(best, candidate (p, c))

// Exact 64-bit form (any metric): packed (key, label), table entries
// {x | y << 16, x^2 + y^2}.
template <int METRIC, bool COH, bool DEDUP = false>
struct Quad {
  static constexpr bool kDedup = DEDUP;
  static constexpr bool kFillOwn = false;
  long long b[4];
  int m2x, m2y, x0, y;
  const int2* __restrict__ table;
  __device__ __forceinline__ Quad(const PassArgs& a, int x0_, int y_)
      : m2x(-2 * x0_), m2y(-2 * y_), x0(x0_), y(y_), table(a.table) {}
  __device__ __forceinline__ int2 pos(int c) const {
    const int2 e = COH ? __ldca(&table[c]) : __ldg(&table[c]);
    const int sx = e.x & 0xFFFF;
    const int sy = static_cast<int>(static_cast<unsigned int>(e.x) >> 16);
    // the sentinel (c = -1) reads {0, INT32_MAX}: its Euclidean key is
    // INT32_MAX, its Manhattan key 2^30 + x, both above every real key
    if (METRIC == kManhattan) return make_int2(sx, c < 0 ? 0x40000000 : abs(sy - y));
    return make_int2(sx, static_cast<int>(static_cast<uint32_t>(e.y) + static_cast<uint32_t>(m2y) *
                                                                         static_cast<uint32_t>(sy)));
  }
  __device__ __forceinline__ long long key(int i, int2 p, int c) const {
    if (METRIC == kManhattan) return pack_key(abs(p.x - (x0 + i)) + p.y, c);
    return pack_key(static_cast<int>(static_cast<uint32_t>(p.y) +
                                     static_cast<uint32_t>(m2x - 2 * i) * static_cast<uint32_t>(p.x)),
                    c);
  }
  __device__ __forceinline__ void set(int i, int2 p, int c) { b[i] = key(i, p, c); }
  __device__ __forceinline__ void fold(int i, int2 p, int c) { b[i] = min(b[i], key(i, p, c)); }
};

// Clamped 32-bit form (Euclidean): key = min(d^2, cap) * 2^lb + label, with
// cap = 2^(32 - lb) - 1 and every label below 2^lb.  For any pixel whose best
// candidate lies below distance^2 cap - 1 this orders the candidates exactly
// as the 64-bit form (distance, then lowest label), with one 32-bit minimum
// and one clamp instead of the 64-bit compare-and-select.  An empty label
// reads the far position, clamps to cap and (the label wrapping to -1)
// encodes as (cap - 1, 2^lb - 1): a quad whose best reaches cap - 1 is
// recomputed with the exact form, so the result never depends on the cap.
// Prepared position: {s.x, (s.y - y)^2}.
template <bool COH, bool DEDUP = false>
struct Quad32 {
  static constexpr bool kDedup = DEDUP;
  static constexpr bool kFillOwn = false;
  uint32_t b[4];
  int x0, y;
  uint32_t cap, mul;
  const uint32_t* __restrict__ ptable;
  __device__ __forceinline__ Quad32(const PassArgs& a, int x0_, int y_)
      : x0(x0_), y(y_), cap(a.cap), mul(a.mul), ptable(a.ptable) {}
  __device__ __forceinline__ int2 pos(int c) const {
    const uint32_t e = COH ? __ldca(&ptable[c]) : __ldg(&ptable[c]);
    const uint32_t dy = static_cast<uint32_t>(static_cast<int>(e >> 16) - y);
    return make_int2(static_cast<int>(e & 0xFFFFu), static_cast<int>(dy * dy));
  }
  __device__ __forceinline__ uint32_t key(int i, int2 p, int c) const {
    const uint32_t dx = static_cast<uint32_t>(p.x - (x0 + i));
    const uint32_t d = dx * dx + static_cast<uint32_t>(p.y);
    return min(d, cap) * mul + static_cast<uint32_t>(c);
  }
  __device__ __forceinline__ void set(int i, int2 p, int c) { b[i] = key(i, p, c); }
  __device__ __forceinline__ void fold(int i, int2 p, int c) { b[i] = min(b[i], key(i, p, c)); }
};

// Manhattan 32-bit forms: distances are at most 2 * 32767 < 2^17, so with
// every label below 2^lb, lb <= 15, key = d * 2^lb + label is exact without a
// cap.  Prepared position: {s.x, |s.y - y|}; an empty label takes the far
// position's x (kFarX) and the y-term kManhattanFarY, which puts it at
// distance [81919, 114686] from every pixel: above every real distance, below
// 2^17, and (its label wrapping to -1) at a key of at least
// (kManhattanMax + 1) * 2^lb, so a pixel whose best is such a key has no
// candidate at all.  With more labels (CAP) the key is clamped like the
// Euclidean one, min(d, cap) * 2^lb + label with cap = 2^(32 - lb) - 1 <
// 81919, and a quad whose best reaches cap - 1 is recomputed exactly.
constexpr uint32_t kManhattanMax = 2u * 32767u;
constexpr int kManhattanFarY = 65535;

template <bool COH, bool DEDUP = false, bool CAP = false>
struct Quad32M {
  static constexpr bool kDedup = DEDUP;
  static constexpr bool kFillOwn = false;
  uint32_t b[4];
  int x0, y;
  uint32_t cap, mul;
  const uint32_t* __restrict__ ptable;
  __device__ __forceinline__ Quad32M(const PassArgs& a, int x0_, int y_)
      : x0(x0_), y(y_), cap(a.cap), mul(a.mul), ptable(a.ptable) {}
  __device__ __forceinline__ int2 pos(int c) const {
    const uint32_t e = COH ? __ldca(&ptable[c]) : __ldg(&ptable[c]);
    const int ady = c < 0 ? kManhattanFarY : abs(static_cast<int>(e >> 16) - y);
    return make_int2(static_cast<int>(e & 0xFFFFu), ady);
  }
  __device__ __forceinline__ uint32_t key(int i, int2 p, int c) const {
    const uint32_t d = static_cast<uint32_t>(abs(p.x - (x0 + i)) + p.y);
    return (CAP ? min(d, cap) : d) * mul + static_cast<uint32_t>(c);
  }
  __device__ __forceinline__ void set(int i, int2 p, int c) { b[i] = key(i, p, c); }
  __device__ __forceinline__ void fold(int i, int2 p, int c) { b[i] = min(b[i], key(i, p, c)); }
};

// Byte-offset 32-bit form (Euclidean, fewer than 2^16 seeds).  For a seed's
// packed position e = x | y << 16 and a pixel (x_p, y_p),
// v = e - (x_p | y_p << 16) + 2^15 equals (dx + 2^15) + dy * 2^16 with no
// borrow between the halves, so bytes 0 and 2 of v are dx and dy modulo 256,
// and one dp4a of v with those two bytes gives dx^2 + dy^2, exact while both
// lie in [-128, 127].  The gathered entry is used as it is: no unpacking per
// gather.  key = d * 2^16 + label: an empty label (-1) leaves all ones in
// the label field, which names no seed.  Inside the window dx, dy in [-128, 128)
// every key is exact (d <= 2^15); outside it a key may be anything.  After
// the fold each pixel's winner is looked up again: when it lies in its
// pixel's window at d < 128^2, every seed outside the window (at d >= 128^2)
// loses to it and every seed inside was scored exactly, so the winner is the
// exact one; a quad where any pixel fails this is recomputed with the
// clamped form.  The prepared position is e itself.  PRMT packs the key with
// one byte permute (integer ALU pipe) instead of a multiply-add (FMA pipe):
// faster for the k = 1, 2 passes, slower for the others (GB300).  The wide
// form (2^16 seeds and more) widens the label field to lb bits with 2^lb > n
// and narrows the window to the largest power of two h with
// (2h^2 + 1) * 2^lb <= 2^32 (h = 8 at 2^22 seeds), so that no key inside it
// wraps; the same argument then holds with h in place of 128.
constexpr uint32_t kByteWindow = 128;  // h: dx, dy in [-h, h)

template <bool COH, bool DEDUP = false, bool PRMT = false>
struct Quad8 {
  static constexpr bool kDedup = DEDUP;
  // an out-of-range side candidate is replaced by the same row's label at the
  // pixel itself (a candidate the pixel scores anyway) instead of the empty
  // label, whose key is arbitrary in this form
  static constexpr bool kFillOwn = true;
  uint32_t b[4];
  int x0, y;
  uint32_t k0, mul;
  const uint32_t* __restrict__ ptable;
  __device__ __forceinline__ Quad8(const PassArgs& a, int x0_, int y_)
      : x0(x0_),
        y(y_),
        k0(0x8000u - (static_cast<uint32_t>(x0_) + (static_cast<uint32_t>(y_) << 16))),
        mul(a.bmul),  // 2^16
        ptable(a.ptable) {}
  __device__ __forceinline__ int2 pos(int c) const {
    const uint32_t e = COH ? __ldca(&ptable[c]) : __ldg(&ptable[c]);
    return make_int2(static_cast<int>(e), 0);
  }
  __device__ __forceinline__ uint32_t key(int i, int2 p, int c) const {
    const uint32_t v = static_cast<uint32_t>(p.x) + k0 - static_cast<uint32_t>(i);
    const int d = __dp4a(static_cast<int>(v), static_cast<int>(v & 0x00FF00FFu), 0);
    if (PRMT) return __byte_perm(static_cast<uint32_t>(c), static_cast<uint32_t>(d), 0x5410);
    return static_cast<uint32_t>(d) * mul + static_cast<uint32_t>(c);
  }
  __device__ __forceinline__ void set(int i, int2 p, int c) { b[i] = key(i, p, c); }
  __device__ __forceinline__ void fold(int i, int2 p, int c) { b[i] = min(b[i], key(i, p, c)); }
};

// Prepared positions of a label vector.  With Q::kDedup a label equal to its
// left neighbour in the vector reuses that gather: lanes whose quads lie
// inside one cell then issue no table load, which pays when cells are small
// (the table falls out of L1 and most quads straddle a cell boundary) and
// costs issue slots when cells are large.
template <class Q>
__device__ __forceinline__ void gather4(const Q& q, const int4& L, int2 (&p)[4]) {
  p[0] = q.pos(L.x);
  if (Q::kDedup) {
    p[1] = p[0];
    if (L.y != L.x) p[1] = q.pos(L.y);
    p[2] = p[1];
    if (L.z != L.y) p[2] = q.pos(L.z);
    p[3] = p[2];
    if (L.w != L.z) p[3] = q.pos(L.w);
  } else {
    p[1] = q.pos(L.y);
    p[2] = q.pos(L.z);
    p[3] = q.pos(L.w);
  }
}

template <class Q>
__device__ __forceinline__ void init4(Q& q, const int4& L, const int2 (&p)[4]) {
  q.set(0, p[0], L.x);
  q.set(1, p[1], L.y);
  q.set(2, p[2], L.z);
  q.set(3, p[3], L.w);
}

template <class Q>
__device__ __forceinline__ void fold4(Q& q, const int4& L, const int2 (&p)[4]) {
  q.fold(0, p[0], L.x);
  q.fold(1, p[1], L.y);
  q.fold(2, p[2], L.z);
  q.fold(3, p[3], L.w);
}

// Pixel x0 + i takes label L_i (i = 0..3).
template <class Q>
__device__ __forceinline__ void fold4(Q& q, const int4& L) {
  int2 p[4];
  gather4(q, L, p);
  fold4(q, L, p);
}

// Labels at columns x0 + dx .. x0 + dx + 3 of one row for |dx| = k, a multiple
// of 4 (one aligned 16-byte load); columns outside [0, pitch) read as -1 and
// the row padding [w, pitch) holds -1 already.
// IN: the quad's block lies inside the map with all its neighbours (no test).
template <bool COH, bool IN = false>
__device__ __forceinline__ int4 load_side(const int32_t* __restrict__ row, int x0, int dx, int pitch,
                                          const int4& fill) {
  const int xs = x0 + dx;
  if (IN) return map4<COH>(row + xs);
  return (xs >= 0 && xs < pitch) ? map4<COH>(row + xs) : fill;
}

template <bool COH>
__device__ __forceinline__ int4 load_scalar4(const int32_t* __restrict__ row, int xs, int w, const int4& fill) {
  const int f[4] = {fill.x, fill.y, fill.z, fill.w};
  int v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = (xs + i >= 0 && xs + i < w) ? map1<COH>(row + xs + i) : f[i];
  return make_int4(v[0], v[1], v[2], v[3]);
}

// The side candidates (x -/+ k) of one source row for the four pixels of a
// thread; `mid` is that row's vector at x0 and `mp` its prepared positions.
// For k = 1 and k = 2 the side labels of neighbouring pixels overlap the
// row's own vector: only the 2 (k = 1) or 4 (k = 2) labels outside it are
// gathered, and the 8 side candidates reuse `mp` for the rest.
template <int KSEL, bool COH, bool IN = false, class Q>
__device__ __forceinline__ void fold_sides(Q& q, const int32_t* __restrict__ row, const int4& mid,
                                           const int2 (&mp)[4], const PassArgs& a) {
  const int x0 = q.x0;
  // out-of-range candidates: the empty label, or (Q::kFillOwn) the row's own
  // label at the pixel, which that pixel scores anyway
  const int4 fill = Q::kFillOwn ? mid : make_int4(-1, -1, -1, -1);
  if (KSEL == 0) {
    const int4 L = load_side<COH, IN>(row, x0, -a.k, a.pitch, fill);
    const int4 R = load_side<COH, IN>(row, x0, a.k, a.pitch, fill);
    fold4(q, L);
    group_fence();
    fold4(q, R);
  } else if (KSEL == 1) {
    // left of pixel i: column x0 + i - 1; right: x0 + i + 1
    const int l = (IN || x0 >= 4) ? map1<COH>(row + x0 - 1) : fill.x;
    const int r = (IN || x0 + 4 < a.pitch) ? map1<COH>(row + x0 + 4) : fill.w;
    const int2 pl = q.pos(l);
    const int2 pr = q.pos(r);
    q.fold(0, pl, l);
    q.fold(1, mp[0], mid.x);
    q.fold(2, mp[1], mid.y);
    q.fold(3, mp[2], mid.z);
    q.fold(0, mp[1], mid.y);
    q.fold(1, mp[2], mid.z);
    q.fold(2, mp[3], mid.w);
    q.fold(3, pr, r);
  } else if (KSEL == 2) {
    // left of pixel i: column x0 + i - 2; right: x0 + i + 2
    const int2 l = (IN || x0 >= 4) ? map2<COH>(row + x0 - 2) : make_int2(fill.x, fill.y);
    const int2 r = (IN || x0 + 4 < a.pitch) ? map2<COH>(row + x0 + 4) : make_int2(fill.z, fill.w);
    const int2 pl0 = q.pos(l.x);
    const int2 pl1 = q.pos(l.y);
    const int2 pr0 = q.pos(r.x);
    const int2 pr1 = q.pos(r.y);
    q.fold(0, pl0, l.x);
    q.fold(1, pl1, l.y);
    q.fold(2, mp[0], mid.x);
    q.fold(3, mp[1], mid.y);
    q.fold(0, mp[2], mid.z);
    q.fold(1, mp[3], mid.w);
    q.fold(2, pr0, r.x);
    q.fold(3, pr1, r.y);
  } else {
    const int4 L = load_scalar4<COH>(row, x0 - a.k, a.w, fill);
    const int4 R = load_scalar4<COH>(row, x0 + a.k, a.w, fill);
    fold4(q, L);
    group_fence();
    fold4(q, R);
  }
  group_fence();
}

// One jump pass (Table I / Section V-B) for the four horizontally adjacent
// pixels (x0 .. x0+3, y) of one thread: it starts from their own labels and
// folds in the neighbour offsets one source row at a time (16-byte label
// loads, seed gathers and minimums).  Candidate order does not matter: every
// key form is a total order.
template <int NB, int KSEL, bool COH, bool IN = false, class Q>
__device__ __forceinline__ void fold_all(Q& q, const PassArgs& a, int x0, int y) {
  const int64_t pitch = a.pitch;
  const int32_t* crow = a.src + y * pitch;
  const int4 own = map4<COH>(crow + x0);
  // the first up-row vector is in flight while the own labels are scored
  const bool up_ok = IN || y - a.k >= 0;
  const bool dn_ok = IN || y + a.k < a.h;
  const int32_t* urow = a.src + (y - a.k) * pitch;
  const int32_t* drow = a.src + (y + a.k) * pitch;
  const int4 neg = make_int4(-1, -1, -1, -1);
  const int4 um = up_ok ? map4<COH>(urow + x0) : neg;
  int2 p[4];
  gather4(q, own, p);
  init4(q, own, p);
  group_fence();
  // centre row: (-k, 0), (+k, 0)
  fold_sides<KSEL, COH, IN>(q, crow, own, p, a);
  // up row: (0, -k) and, for Moore, (-k, -k), (+k, -k); then the down row
  if (up_ok) {
    const int4 dm = dn_ok ? map4<COH>(drow + x0) : neg;
    gather4(q, um, p);
    fold4(q, um, p);
    group_fence();
    if (NB == kMoore) fold_sides<KSEL, COH, IN>(q, urow, um, p, a);
    if (dn_ok) {
      gather4(q, dm, p);
      fold4(q, dm, p);
      group_fence();
      if (NB == kMoore) fold_sides<KSEL, COH, IN>(q, drow, dm, p, a);
    }
  } else if (dn_ok) {
    const int4 dm = map4<COH>(drow + x0);
    gather4(q, dm, p);
    fold4(q, dm, p);
    group_fence();
    if (NB == kMoore) fold_sides<KSEL, COH, IN>(q, drow, dm, p, a);
  }
}

template <bool IN = false>
__device__ __forceinline__ void store_quad(const PassArgs& a, int x0, int y, int l0, int l1, int l2, int l3) {
  int4 out;
  out.x = (IN || x0 < a.w) ? l0 : -1;
  out.y = (IN || x0 + 1 < a.w) ? l1 : -1;
  out.z = (IN || x0 + 2 < a.w) ? l2 : -1;
  out.w = (IN || x0 + 3 < a.w) ? l3 : -1;
  *reinterpret_cast<int4*>(a.dst + static_cast<int64_t>(y) * a.pitch + x0) = out;
}

__device__ __forceinline__ int low_label(long long b) { return static_cast<int>(static_cast<unsigned int>(b)); }

// Exact form (any metric).
template <int NB, int METRIC, int KSEL, bool COH = false, bool DEDUP = false, bool IN = false>
__device__ __forceinline__ void pass_quad(const PassArgs& a, int x0, int y) {
  Quad<METRIC, COH, DEDUP> q(a, x0, y);
  fold_all<NB, KSEL, COH, IN>(q, a, x0, y);
  store_quad<IN>(a, x0, y, low_label(q.b[0]), low_label(q.b[1]), low_label(q.b[2]), low_label(q.b[3]));
}

// 32-bit forms.  Euclidean, and Manhattan with MCAP (more than 2^15 labels):
// clamped, falling back to the exact form for a quad whose best distance
// reaches the cap (or that saw only empty labels).  Manhattan without MCAP:
// exact as is (lb <= 15); an all-empty pixel stays -1.
template <int NB, int KSEL, bool COH = false, int METRIC = kEuclid, bool DEDUP = false, bool MCAP = false,
          bool IN = false>
__device__ __forceinline__ void pass_quad_clamped(const PassArgs& a, int x0, int y) {
  const uint32_t mask = a.mul - 1u;
  if (METRIC == kManhattan && MCAP) {
    Quad32M<COH, DEDUP, true> q(a, x0, y);
    fold_all<NB, KSEL, COH, IN>(q, a, x0, y);
    const uint32_t lim = (a.cap - 1u) * a.mul;
    if (max(max(q.b[0], q.b[1]), max(q.b[2], q.b[3])) >= lim) {
      pass_quad<NB, kManhattan, KSEL, COH, DEDUP, IN>(a, x0, y);
      return;
    }
    store_quad<IN>(a, x0, y, static_cast<int>(q.b[0] & mask), static_cast<int>(q.b[1] & mask),
               static_cast<int>(q.b[2] & mask), static_cast<int>(q.b[3] & mask));
    return;
  }
  if (METRIC == kManhattan) {
    Quad32M<COH, DEDUP> q(a, x0, y);
    fold_all<NB, KSEL, COH, IN>(q, a, x0, y);
    const uint32_t lim = (kManhattanMax + 1u) * a.mul;
    store_quad<IN>(a, x0, y, q.b[0] >= lim ? -1 : static_cast<int>(q.b[0] & mask),
               q.b[1] >= lim ? -1 : static_cast<int>(q.b[1] & mask),
               q.b[2] >= lim ? -1 : static_cast<int>(q.b[2] & mask),
               q.b[3] >= lim ? -1 : static_cast<int>(q.b[3] & mask));
    return;
  }
  Quad32<COH, DEDUP> q(a, x0, y);
  fold_all<NB, KSEL, COH, IN>(q, a, x0, y);
  const uint32_t lim = (a.cap - 1u) * a.mul;
  if (max(max(q.b[0], q.b[1]), max(q.b[2], q.b[3])) >= lim) {
    pass_quad<NB, kEuclid, KSEL, COH, DEDUP, IN>(a, x0, y);
    return;
  }
  store_quad<IN>(a, x0, y, static_cast<int>(q.b[0] & mask), static_cast<int>(q.b[1] & mask),
             static_cast<int>(q.b[2] & mask), static_cast<int>(q.b[3] & mask));
}

// The byte-offset form's recomputation, out of line: it is rare, and kept
// apart it leaves the common path the registers of the byte form alone.
template <int NB, int KSEL, bool COH, bool DEDUP>
__device__ __noinline__ void byte_fallback(const PassArgs a, int x0, int y) {
  pass_quad_clamped<NB, KSEL, COH, kEuclid, DEDUP>(a, x0, y);
}

// Byte-offset form (Euclidean): the fold, then the winner check described at
// Quad8; a quad that fails it is recomputed with the clamped form.
template <int NB, int KSEL, bool COH = false, bool DEDUP = false, bool WIDE = false, bool IN = false>
__device__ __forceinline__ void pass_quad_byte(const PassArgs& a, int x0, int y) {
  Quad8<COH, DEDUP, !WIDE && KSEL != 0> q(a, x0, y);
  fold_all<NB, KSEL, COH, IN>(q, a, x0, y);
  // packed positions with the far position first: the label field plus one,
  // masked, indexes it (all ones, an empty label, wraps to the far position)
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
    const uint32_t e = COH ? __ldca(&arena[j]) : __ldg(&arena[j]);
    // (dx + h) | (dy + h) << 16 has no bit at or above 2h in either half
    // exactly when dx, dy lie in [-h, h)
    bad |= (e + kw - static_cast<uint32_t>(i)) & wmask;
  }
  const uint32_t top = max(max(q.b[0], q.b[1]), max(q.b[2], q.b[3]));
  if (bad != 0 || top >= (WIDE ? a.blim : (h * h) << 16)) {
    byte_fallback<NB, KSEL, COH, DEDUP>(a, x0, y);
    return;
  }
  store_quad<IN>(a, x0, y, static_cast<int>(q.b[0] & mask), static_cast<int>(q.b[1] & mask),
                 static_cast<int>(q.b[2] & mask), static_cast<int>(q.b[3] & mask));
}

// Pass launch shape: 128-thread blocks (64 quads x 2 rows on wide maps), 10
// resident per SM, which leaves 48 registers a thread: measured on the GB300
// against 256-thread blocks at 40 and 64 registers, and 64-thread blocks, this
// is the fastest on every map size tried (1024^2 .. 8192^2).
constexpr int kPassThreads = 128;
#ifndef VD_PASS_MIN_BLOCKS
#define VD_PASS_MIN_BLOCKS 10
#endif

// The byte-offset form needs fewer registers: 16 blocks (32 registers a
// thread, full occupancy) measured faster than 10 and 12 on the GB300; its
// rare recomputation (byte_fallback) spills at that budget.
#ifndef VD_BYTE_MIN_BLOCKS
#define VD_BYTE_MIN_BLOCKS 16
#endif

// KEY: 0 the exact 64-bit form, 1 the 32-bit form of METRIC, 2 the clamped
// Manhattan 32-bit form (more than 2^15 labels), 3 the Euclidean byte-offset
// form, 4 its wide form (2^16 seeds and more).
template <int NB, int METRIC, int KSEL, int KEY = 0, bool DEDUP = false>
__global__ void __launch_bounds__(kPassThreads, KEY >= 3 ? VD_BYTE_MIN_BLOCKS : VD_PASS_MIN_BLOCKS)
    k_pass(PassArgs a) {
  pdl_trigger();
  pdl_wait();
  const int x0 = 4 * static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
  int rb = blockIdx.y;
  if (a.band_m > 1) rb = (blockIdx.y % a.band_t) * a.band_m + blockIdx.y / a.band_t;
  const int yb = a.y0 + rb * static_cast<int>(blockDim.y);
  const int y = yb + static_cast<int>(threadIdx.y);
  if (x0 >= a.pitch || y >= a.y_end) return;
  // a block whose pixels lie in the map, away from its edges by k in both
  // directions, reads every neighbour inside the map: no range tests (the
  // test is uniform across the block, so the two paths never diverge a warp)
  const int xb = 4 * static_cast<int>(blockIdx.x * blockDim.x);
  const bool in = KSEL <= 2 && xb - a.k >= 0 && xb + 4 * static_cast<int>(blockDim.x) + a.k <= a.w &&
                  yb - a.k >= 0 && yb + static_cast<int>(blockDim.y) + a.k <= a.h &&
                  yb + static_cast<int>(blockDim.y) <= a.y_end;
  if (in) {
    if (KEY == 3 || KEY == 4) pass_quad_byte<NB, KSEL, false, DEDUP, KEY == 4, true>(a, x0, y);
    else if (KEY != 0) pass_quad_clamped<NB, KSEL, false, METRIC, DEDUP, KEY == 2, true>(a, x0, y);
    else pass_quad<NB, METRIC, KSEL, false, DEDUP, true>(a, x0, y);
    return;
  }
  if (KEY == 3 || KEY == 4) pass_quad_byte<NB, KSEL, false, DEDUP, KEY == 4>(a, x0, y);
  else if (KEY != 0) pass_quad_clamped<NB, KSEL, false, METRIC, DEDUP, KEY == 2>(a, x0, y);
  else pass_quad<NB, METRIC, KSEL, false, DEDUP>(a, x0, y);
}

// ---------------------------------------------------------------------------
// Fused group of small-step passes in shared memory.
// ---------------------------------------------------------------------------

constexpr int kMaxFused = 8;

struct FusedArgs {
  const int32_t* __restrict__ src;
  int32_t* __restrict__ dst;
  const int2* __restrict__ table;  // entry -1 is the sentinel
  uint32_t n_seeds;
  int w, h, pitch;
  int n_pass;
  int ks[kMaxFused];
  int nbs[kMaxFused];
  int halo;      // sum of ks
  int tx, ty;    // output tile
};

// A tile of (tx + 2 halo) x (ty + 2 halo) labels is loaded once; pass j then
// recomputes the tile grown by the steps still to come, so its neighbours at
// offset k_j always lie inside the region the previous pass produced.
// Out-of-grid cells hold -1 in every pass, exactly as an unfused pass skips
// out-of-grid neighbours, so the result equals the unfused passes bit for bit.
template <int METRIC>
__global__ void __launch_bounds__(256) k_pass_fused(FusedArgs a) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ int32_t smem[];
  const int H = a.halo;
  const int SW = a.tx + 2 * H;
  const int SH = a.ty + 2 * H;
  int32_t* A = smem;
  int32_t* B = smem + SW * SH;
  const int gx0 = static_cast<int>(blockIdx.x) * a.tx - H;  // grid coords of smem (0, 0)
  const int gy0 = static_cast<int>(blockIdx.y) * a.ty - H;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int bx = blockDim.x, by = blockDim.y;
  const int64_t pitch = a.pitch;

  for (int sy = ty; sy < SH; sy += by) {
    const int gy = gy0 + sy;
    const bool row_ok = gy >= 0 && gy < a.h;
    const int32_t* row = a.src + (row_ok ? gy : 0) * pitch;
    for (int sx = tx; sx < SW; sx += bx) {
      const int gx = gx0 + sx;
      A[sy * SW + sx] = (row_ok && gx >= 0 && gx < a.w) ? __ldg(row + gx) : -1;
    }
  }
  __syncthreads();

  int rem = H;
  for (int p = 0; p < a.n_pass; ++p) {
    const int k = a.ks[p];
    const bool moore = a.nbs[p] == kMoore;
    rem -= k;
    const int lo = H - rem;            // first smem row/col of this pass's region
    const int rw = a.tx + 2 * rem;
    const int rh = a.ty + 2 * rem;
    for (int ry = ty; ry < rh; ry += by) {
      const int sy = lo + ry;
      const int y = gy0 + sy;
      for (int rx = tx; rx < rw; rx += bx) {
        const int sx = lo + rx;
        const int x = gx0 + sx;
        int res = -1;
        if (x >= 0 && x < a.w && y >= 0 && y < a.h) {
          const int32_t* c = A + sy * SW + sx;
          const int m2x = -2 * x, m2y = -2 * y;
          long long b = cand<METRIC>(c[0], a.table, m2x, m2y, x, y);
          b = fold<METRIC>(b, c[k], a.table, m2x, m2y, x, y);
          b = fold<METRIC>(b, c[-k], a.table, m2x, m2y, x, y);
          b = fold<METRIC>(b, c[k * SW], a.table, m2x, m2y, x, y);
          b = fold<METRIC>(b, c[-k * SW], a.table, m2x, m2y, x, y);
          if (moore) {
            b = fold<METRIC>(b, c[k * SW + k], a.table, m2x, m2y, x, y);
            b = fold<METRIC>(b, c[k * SW - k], a.table, m2x, m2y, x, y);
            b = fold<METRIC>(b, c[-k * SW - k], a.table, m2x, m2y, x, y);
            b = fold<METRIC>(b, c[-k * SW + k], a.table, m2x, m2y, x, y);
          }
          res = static_cast<int>(static_cast<unsigned int>(b));
        }
        B[sy * SW + sx] = res;
      }
    }
    __syncthreads();
    int32_t* t = A;
    A = B;
    B = t;
  }

  // write the tile (columns up to the pitch, so the padding stays -1)
  for (int ry = ty; ry < a.ty; ry += by) {
    const int y = gy0 + H + ry;
    if (y >= a.h) break;
    for (int rx = tx; rx < a.tx; rx += bx) {
      const int x = gx0 + H + rx;
      if (x < a.pitch) a.dst[y * pitch + x] = (x < a.w) ? A[(H + ry) * SW + H + rx] : -1;
    }
  }
}

// ---------------------------------------------------------------------------
// Seeds: move, stamp
// ---------------------------------------------------------------------------

// SplitMix64 (Steele, Lea, Flood 2014): n-th output of the generator started
// at `state`.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t state, uint64_t n) {
  uint64_t z = state + (n + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int rng_disp(uint64_t key, uint64_t step, uint64_t k, int axis, int max_disp) {
  const uint64_t draw = splitmix64(key, (step << 33) + 2 * k + static_cast<uint64_t>(axis));
  const uint64_t m = static_cast<uint64_t>(2 * max_disp + 1);
  return static_cast<int>(((draw >> 32) * m) >> 32) - max_disp;
}

// Rebuilds the pass tables (entry k + 1 for seed k; entry 0 the sentinels).
static __global__ void k_build_table(const int2* __restrict__ seeds, int n, int2* __restrict__ table,
                                     uint32_t* __restrict__ ptable) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    table[0] = make_int2(0, kSentinelNorm);
    ptable[0] = pack_pos(static_cast<int>(kFarX), 0);
  }
  if (k < n) {
    const int2 p = seeds[k];
    table[k + 1] = table_entry(p);
    ptable[k + 1] = pack_pos(p.x, p.y);
  }
}

// Flags any label outside [-1, n) (device-side input validation).
static __global__ void k_check_labels(const int32_t* __restrict__ labels, int64_t count, int n,
                               unsigned long long* __restrict__ bad) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = labels[i];
    if (l < -1 || l >= n) atomicAdd(bad, 1ULL);
  }
}

struct MoveArgs {
  int2* seeds;
  int2* table;
  uint32_t* ptable;
  int n;
  const int2* dxy;  // given displacements, or null: SplitMix64 draws in [-max_disp, max_disp]
  int w, h, max_disp;
  uint64_t key, step;
};

// SimulateParticles (Algorithm 1): p_k <- clamp(p_k + delta_k) on the grid;
// also refreshes the seed's pass-table entries.
static __global__ void k_move(MoveArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  int2 p = a.seeds[k];
  long long dx, dy;
  if (a.dxy != nullptr) {
    const int2 d = a.dxy[k];
    dx = d.x;
    dy = d.y;
  } else {
    dx = rng_disp(a.key, a.step, static_cast<uint64_t>(k), 0, a.max_disp);
    dy = rng_disp(a.key, a.step, static_cast<uint64_t>(k), 1, a.max_disp);
  }
  long long x = p.x + dx, y = p.y + dy;
  x = x < 0 ? 0 : (x > a.w - 1 ? a.w - 1 : x);
  y = y < 0 ? 0 : (y > a.h - 1 ? a.h - 1 : y);
  p.x = static_cast<int>(x);
  p.y = static_cast<int>(y);
  a.seeds[k] = p;
  a.table[k + 1] = table_entry(p);
  a.ptable[k + 1] = pack_pos(p.x, p.y);
}

// The stamp on a map with stale labels (reading R4: each seed pixel gets the
// lowest index standing on it; the rest of the map is kept), one random
// access a seed: seed k swaps itself into its pixel and, when the label it
// took out is a lower index r whose seed stands on the same pixel, puts r
// back with an atomic minimum.  Every seed at the pixel swaps once, so after
// the last write of the lowest of them, m, any later swap takes m out and
// its seed writes m back: the pixel ends at m.  (A stale label or an empty
// one is dropped; the positions are the move's, read after it completed.)
// It replaces an overwrite of every seed pixel followed by an atomic minimum
// on each: two rounds of scattered sector read-modify-writes in DRAM instead
// of one (8192^2 with 2^22 seeds: 0.28 ms a frame for the two).  With pk_m
// it also writes the seed entries of the position-tagged passes, as
// k_stamp_min.
__device__ __forceinline__ void stamp_seed_entries(int k, int2 p, uint2* __restrict__ pkf,
                                                   const uint32_t* __restrict__ parena, int pk_m) {
  // the word bits of layout pk_m: wide, bit 24 set, x mod 2^m at
  // [24 - m, 24), y mod 2^m at [32 - m, 32); split (m = 4), label bits
  // 20-21 at [24, 26), bit 26 set, x mod 16 at [20, 24), y mod 16 at [28, 32)
  const uint32_t xm = (1u << pk_m) - 1u;
  const uint32_t f =
      pk_m == 4 ? ((static_cast<uint32_t>(k) & 0x300000u) << 4) | (1u << 26) |
                      ((static_cast<uint32_t>(p.x) & 15u) << 20) | ((static_cast<uint32_t>(p.y) & 15u) << 28)
                : (1u << 24) | ((static_cast<uint32_t>(p.x) & xm) << (24 - pk_m)) |
                      ((static_cast<uint32_t>(p.y) & xm) << (32 - pk_m));
  pkf[k + 1] = make_uint2(pack_pos(p.x, p.y), f);
  if (k == 0) pkf[0] = make_uint2(parena[0], 0u);
}

static __global__ void k_stamp_xchg(int32_t* __restrict__ labels, int pitch, const int2* __restrict__ seeds, int n,
                                    uint2* __restrict__ pkf, const uint32_t* __restrict__ parena, int pk_m) {
  pdl_trigger();
  pdl_wait();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 p = seeds[k];
  unsigned int* px = reinterpret_cast<unsigned int*>(labels + static_cast<int64_t>(p.y) * pitch + p.x);
  const int r = static_cast<int>(atomicExch(px, static_cast<unsigned int>(k)));
  if (r >= 0 && r < k) {
    const int2 q = seeds[r];
    if (q.x == p.x && q.y == p.y) atomicMin(px, static_cast<unsigned int>(r));
  }
  if (pk_m) stamp_seed_entries(k, p, pkf, parena, pk_m);
}

// The stamp on an emptied map: the lowest index standing on the pixel wins
// (as unsigned, -1 is the largest value).  With pk_m = 6, 7 or 4 it also
// writes the frame's entries of the position-tagged passes' seed table (pkf:
// n + 1 entries {x | y << 16, the seed's word bits but the label's low
// bits}, [0] the far position; parena: the packed positions with the far one
// first): the stamp runs right before every dJFA frame's passes, after the
// move.
static __global__ void k_stamp_min(int32_t* __restrict__ labels, int pitch, const int2* __restrict__ seeds,
                            int n, uint2* __restrict__ pkf, const uint32_t* __restrict__ parena, int pk_m) {
  pdl_trigger();
  pdl_wait();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 p = seeds[k];
  atomicMin(reinterpret_cast<unsigned int*>(labels + static_cast<int64_t>(p.y) * pitch + p.x),
            static_cast<unsigned int>(k));
  if (pk_m) stamp_seed_entries(k, p, pkf, parena, pk_m);
}

static __global__ void k_fill(int4* __restrict__ p, int64_t n4, int v) {
  pdl_trigger();
  pdl_wait();
  const int4 val = make_int4(v, v, v, v);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n4;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = val;
}

// Flags any seed outside the grid (device-side input validation).
static __global__ void k_check_seeds(const int2* __restrict__ seeds, int n, int w, int h,
                              unsigned long long* __restrict__ bad) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 p = seeds[k];
  if (p.x < 0 || p.x >= w || p.y < 0 || p.y >= h) atomicAdd(bad, 1ULL);
}

// ---------------------------------------------------------------------------
// Seed insertion and removal between frames (the paper leaves both to future
// work, Section VII; the rule is this library's: survivors keep their order and
// are renumbered, new seeds follow, a removed seed's pixels become empty)
// ---------------------------------------------------------------------------

static __global__ void k_fill_i32(int* __restrict__ p, int n, int v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}

// keep[id] = 0 for every removed index; an index out of range or listed twice
// is counted in *bad.
static __global__ void k_update_remove(const int* __restrict__ remove, int n_remove, int n, int* __restrict__ keep,
                                       unsigned long long* __restrict__ bad) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_remove) return;
  const int id = remove[j];
  if (id < 0 || id >= n) {
    atomicAdd(bad, 1ULL);
    return;
  }
  if (atomicExch(&keep[id], 0) == 0) atomicAdd(bad, 1ULL);
}

// The new seed array: each survivor at its new index (the exclusive prefix
// sum of keep, newidx[n] = survivors), then the added seeds.
static __global__ void k_update_compact(const int2* __restrict__ seeds, int n, const int* __restrict__ keep,
                                        const int* __restrict__ newidx, const int2* __restrict__ add, int n_add,
                                        int2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    if (keep[i]) out[newidx[i]] = seeds[i];
  } else if (i < n + n_add) {
    out[newidx[n] + (i - n)] = add[i - n];
  }
}

// Relabels a map in place: a surviving seed's label becomes its new index, a
// removed seed's -1; empty pixels and the row padding stay -1.
static __global__ void k_update_relabel(int32_t* __restrict__ labels, int64_t count, const int* __restrict__ keep,
                                        const int* __restrict__ newidx) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < count;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int l = labels[i];
    if (l >= 0) labels[i] = keep[l] ? newidx[l] : -1;
  }
}

// ---------------------------------------------------------------------------
// Similarity counts (Section VI-A)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

template <int METRIC>
__global__ void __launch_bounds__(256) k_similarity(const int32_t* __restrict__ labels, int pitch,
                                                    const int2* __restrict__ seeds, uint32_t n, int w,
                                                    int h, const int32_t* __restrict__ exact,
                                                    int exact_pitch, const int32_t* __restrict__ ref,
                                                    int ref_pitch,
                                                    unsigned long long* __restrict__ counters) {
  unsigned long long ne = 0, nm = 0;
  const int64_t total = static_cast<int64_t>(w) * h;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int y = static_cast<int>(i / w);
    const int x = static_cast<int>(i - static_cast<int64_t>(y) * w);
    const int l = labels[static_cast<int64_t>(y) * pitch + x];
    if (exact != nullptr && static_cast<uint32_t>(l) < n) {
      const uint32_t d = seed_dist<METRIC>(seeds[l], x, y);
      ne += (d == static_cast<uint32_t>(exact[static_cast<int64_t>(y) * exact_pitch + x])) ? 1 : 0;
    }
    if (ref != nullptr) nm += (l == ref[static_cast<int64_t>(y) * ref_pitch + x]) ? 1 : 0;
  }
  __shared__ unsigned long long s_e[8], s_m[8];
  ne = warp_sum(ne);
  nm = warp_sum(nm);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_e[wid] = ne;
    s_m[wid] = nm;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long te = 0, tm = 0;
    for (int j = 0; j < static_cast<int>(blockDim.x >> 5); ++j) {
      te += s_e[j];
      tm += s_m[j];
    }
    if (te) atomicAdd(&counters[0], te);
    if (tm) atomicAdd(&counters[1], tm);
  }
}

// ---------------------------------------------------------------------------
// Exact diagram (Eq. 1) through a uniform bucket grid
// ---------------------------------------------------------------------------

struct Buckets {
  int cell;          // bucket side in pixels
  int gw, gh;        // buckets per row / column
  const int* start;  // gw*gh + 1 offsets into `ids`
  const int* ids;    // seed indices grouped by bucket
};

static __global__ void k_bucket_count(const int2* __restrict__ seeds, int n, int cell, int gw,
                               int* __restrict__ count) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 p = seeds[k];
  atomicAdd(&count[(p.y / cell) * gw + p.x / cell], 1);
}

static __global__ void k_bucket_fill(const int2* __restrict__ seeds, int n, int cell, int gw,
                              const int* __restrict__ start, int* __restrict__ cursor,
                              int* __restrict__ ids) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 p = seeds[k];
  const int b = (p.y / cell) * gw + p.x / cell;
  ids[start[b] + atomicAdd(&cursor[b], 1)] = k;
}

// Exclusive scan of `count` (length m) into `start` (length m + 1), one
// block of 1024 threads walking the array in chunks with a running carry.
static __global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ count, int m,
                                               int* __restrict__ start) {
  __shared__ int s[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < m; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < m ? count[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < m) start[i] = carry + s[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) start[m] = carry;
}

template <int METRIC>
__device__ __forceinline__ void scan_bucket(const Buckets& b, const int2* __restrict__ seeds, int bi,
                                            int x, int y, uint32_t& bd, int& bl) {
  for (int j = b.start[bi]; j < b.start[bi + 1]; ++j) {
    const int c = b.ids[j];
    const uint32_t d = seed_dist<METRIC>(__ldg(&seeds[c]), x, y);
    if (d < bd || (d == bd && c < bl)) {
      bd = d;
      bl = c;
    }
  }
}

template <int METRIC>
__global__ void __launch_bounds__(256) k_exact(Buckets b, const int2* __restrict__ seeds, int w, int h,
                                               int32_t* __restrict__ out_label,
                                               int32_t* __restrict__ out_dist) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= w || y >= h) return;
  const int cx = x / b.cell, cy = y / b.cell;
  const int ox = x - cx * b.cell, oy = y - cy * b.cell;
  const int edge = min(min(ox, b.cell - 1 - ox), min(oy, b.cell - 1 - oy));
  uint32_t bd = 0xFFFFFFFFu;
  int bl = -1;
  const int rmax = max(b.gw, b.gh);
  for (int r = 0; r <= rmax; ++r) {
    const int y0 = cy - r, y1 = cy + r, x0 = cx - r, x1 = cx + r;
    for (int by = max(y0, 0); by <= min(y1, b.gh - 1); ++by) {
      if (by == y0 || by == y1) {
        for (int bx = max(x0, 0); bx <= min(x1, b.gw - 1); ++bx)
          scan_bucket<METRIC>(b, seeds, by * b.gw + bx, x, y, bd, bl);
      } else {
        if (x0 >= 0) scan_bucket<METRIC>(b, seeds, by * b.gw + x0, x, y, bd, bl);
        if (x1 < b.gw) scan_bucket<METRIC>(b, seeds, by * b.gw + x1, x, y, bd, bl);
      }
    }
    // any seed in ring r+1 or beyond is at least this far along one axis
    const long long lb1 = static_cast<long long>(r) * b.cell + 1 + edge;
    const long long lb = (METRIC == kManhattan) ? lb1 : lb1 * lb1;
    if (bl >= 0 && static_cast<long long>(bd) < lb) break;
  }
  const int64_t i = static_cast<int64_t>(y) * w + x;
  if (out_label) out_label[i] = bl;
  if (out_dist) out_dist[i] = static_cast<int32_t>(bd);
}

}  // namespace vdk
