// vd_pass_pos.cu -- the passes of a JFA frame on a position map.
//
// A JFA frame (Section III, Eq. 2, Table I) floods the seeds over an emptied
// map with steps k_1, k_1 / 2, ..., 1.  In its middle passes neighbouring
// pixels name unrelated, distant seeds, so the plain pass's table gathers
// (one per candidate, nine per pixel) scatter over the whole seed table: on
// the GB300 with 2^18 seeds on 8192^2 those passes are bound by L1 throughput
// at about 28 sectors per warp-wide gather, 4 to 6 times slower than a pass
// over a settled map.  Here the frame's passes with k % 4 == 0 read and write
// a position map instead: each pixel holds (label, packed position
// x | y << 16) of its seed, so a candidate's position arrives with its label
// in the same coalesced load and nothing is gathered; the winner's position
// is looked up once per pixel.  The map is twice as large, so these passes
// move 16 bytes a pixel instead of 8, but stream them.  The last of these
// passes writes the ordinary label map, on which the frame's k = 2 and k = 1
// passes run as usual.  Candidates, distances (exact, 32-bit) and the
// lowest-label tie rule are those of the plain pass, so the labels are
// identical bit for bit.
#include <algorithm>

#include "vd.h"
#include "vd_internal.h"
#include "vd_kernels.cuh"

namespace vdk {

struct PosArgs {
  const int2* __restrict__ src;       // (label, x | y << 16) per pixel; label -1 = empty
  int2* __restrict__ dst;             // next position map, or
  int32_t* __restrict__ dst32;        // the label map (the frame's last position-map pass)
  const uint32_t* __restrict__ ptable;  // packed seed positions
  int w, h, pitch, k;
  int band_m, band_t;
};

// The (distance, label) key of candidate (c, e) for pixel (x, y): exact
// squared Euclidean or Manhattan distance in the high word, the label in the
// low word, so one 64-bit minimum applies the lowest-label tie rule; an empty
// candidate gets the largest key.
template <int METRIC>
__device__ __forceinline__ unsigned long long pos_key(int c, uint32_t e, int x, int y) {
  const int dx = static_cast<int>(e & 0xFFFFu) - x;
  const int dy = static_cast<int>(e >> 16) - y;
  const uint32_t d =
      METRIC == kManhattan ? static_cast<uint32_t>(abs(dx) + abs(dy)) : static_cast<uint32_t>(dx * dx + dy * dy);
  const unsigned long long key = (static_cast<unsigned long long>(d) << 32) | static_cast<uint32_t>(c);
  return c < 0 ? ~0ull : key;
}

template <int METRIC>
__device__ __forceinline__ void pos_fold(unsigned long long (&b)[4], const int4& lo, const int4& hi, int x0, int y) {
  b[0] = min(b[0], pos_key<METRIC>(lo.x, static_cast<uint32_t>(lo.y), x0, y));
  b[1] = min(b[1], pos_key<METRIC>(lo.z, static_cast<uint32_t>(lo.w), x0 + 1, y));
  b[2] = min(b[2], pos_key<METRIC>(hi.x, static_cast<uint32_t>(hi.y), x0 + 2, y));
  b[3] = min(b[3], pos_key<METRIC>(hi.z, static_cast<uint32_t>(hi.w), x0 + 3, y));
}

// One pass with k % 4 == 0 for the quad (x0 .. x0+3, y): its own entries and
// those of the neighbour quads at offset k (Moore, or Von Neumann) that lie
// in the map.  Same launch shape and thread -> quad map as k_pass.
template <int NB, int METRIC, bool OUT32>
__global__ void __launch_bounds__(kPassThreads, VD_PASS_MIN_BLOCKS) k_pass_pos(PosArgs a) {
  pdl_trigger();
  pdl_wait();
  const int x0 = 4 * static_cast<int>(blockIdx.x * blockDim.x + threadIdx.x);
  int rb = blockIdx.y;
  if (a.band_m > 1) rb = (blockIdx.y % a.band_t) * a.band_m + blockIdx.y / a.band_t;
  const int y = rb * static_cast<int>(blockDim.y) + static_cast<int>(threadIdx.y);
  if (x0 >= a.pitch || y >= a.h) return;
  const int64_t pitch = a.pitch;
  const int k = a.k;
  unsigned long long b[4] = {~0ull, ~0ull, ~0ull, ~0ull};
#pragma unroll
  for (int dr = -1; dr <= 1; ++dr) {
    const int yr = y + dr * k;
    if (yr < 0 || yr >= a.h) continue;
    const int2* row = a.src + yr * pitch;
#pragma unroll
    for (int dc = -1; dc <= 1; ++dc) {
      if (NB == kVonNeumann && dr != 0 && dc != 0) continue;
      const int xs = x0 + dc * k;
      if (xs < 0 || xs >= a.pitch) continue;
      const int4 lo = __ldg(reinterpret_cast<const int4*>(row + xs));
      const int4 hi = __ldg(reinterpret_cast<const int4*>(row + xs + 2));
      pos_fold<METRIC>(b, lo, hi, x0, y);
    }
    group_fence();
  }
  int l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) l[i] = (x0 + i < a.w) ? static_cast<int>(static_cast<uint32_t>(b[i])) : -1;
  if (OUT32) {
    *reinterpret_cast<int4*>(a.dst32 + y * pitch + x0) = make_int4(l[0], l[1], l[2], l[3]);
    return;
  }
  uint32_t e[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) e[i] = l[i] >= 0 ? __ldg(&a.ptable[l[i]]) : 0u;
  int4* out = reinterpret_cast<int4*>(a.dst + y * pitch + x0);
  out[0] = make_int4(l[0], static_cast<int>(e[0]), l[1], static_cast<int>(e[1]));
  out[1] = make_int4(l[2], static_cast<int>(e[2]), l[3], static_cast<int>(e[3]));
}

// Empties a position map (label -1 everywhere, row padding included).
static __global__ void k_fill_pos(int4* __restrict__ p, int64_t n4) {
  pdl_trigger();
  pdl_wait();
  const int4 v = make_int4(-1, 0, -1, 0);
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n4;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    p[i] = v;
}

// The stamp on a position map: the lowest index standing on a pixel wins
// (unsigned minimum, under which the empty label -1 is the largest value);
// every seed on the pixel writes the same position.
static __global__ void k_stamp_pos(int2* __restrict__ map, int pitch, const int2* __restrict__ seeds, int n) {
  pdl_trigger();
  pdl_wait();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int2 p = seeds[k];
  int2* px = map + static_cast<int64_t>(p.y) * pitch + p.x;
  atomicMin(reinterpret_cast<unsigned int*>(&px->x), static_cast<unsigned int>(k));
  px->y = static_cast<int>(pack_pos(p.x, p.y));
}

}  // namespace vdk

namespace vdi {

template <typename... KArgs, typename... Args>
static cudaError_t launch_pos_k(void (*kern)(KArgs...), dim3 g, dim3 b, cudaStream_t st, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

int launch_fill_pos(int2* map, int64_t elems, cudaStream_t st, bool pdl) {
  const int64_t n4 = elems / 2;
  const int grid = static_cast<int>(std::min<int64_t>((n4 + 255) / 256, 152 * 16));
  const cudaError_t e = launch_pos_k(vdk::k_fill_pos, dim3(grid), dim3(256), st, pdl, reinterpret_cast<int4*>(map), n4);
  if (e != cudaSuccess) return vd_cuda_check(e, "position map fill");
  return vd_cuda_check(cudaGetLastError(), "position map fill");
}

int launch_stamp_pos(const MapView& m, int2* map, cudaStream_t st, bool pdl) {
  const cudaError_t e =
      launch_pos_k(vdk::k_stamp_pos, dim3((m.n + 255) / 256), dim3(256), st, pdl, map, m.pitch, m.seeds, m.n);
  if (e != cudaSuccess) return vd_cuda_check(e, "position map stamp");
  return vd_cuda_check(cudaGetLastError(), "position map stamp");
}

template <int NB, int METRIC>
static cudaError_t launch_pos_t(bool out32, dim3 g, dim3 b, cudaStream_t st, bool pdl, const vdk::PosArgs& a) {
  if (out32) return launch_pos_k(vdk::k_pass_pos<NB, METRIC, true>, g, b, st, pdl, a);
  return launch_pos_k(vdk::k_pass_pos<NB, METRIC, false>, g, b, st, pdl, a);
}

int launch_pass_pos(const MapView& m, const int2* src, int2* dst, int32_t* dst32, int32_t k, int32_t nb,
                    int32_t metric, int64_t band_min_k, cudaStream_t st, bool pdl) {
  if (k < 4 || k % 4 != 0) return vd_fail(VD_EINVAL, "position-map pass needs k %% 4 == 0, got %d", k);
  vdk::PosArgs a;
  a.src = src;
  a.dst = dst;
  a.dst32 = dst32;
  a.ptable = m.ptable;
  a.w = m.w;
  a.h = m.h;
  a.pitch = m.pitch;
  a.k = k;
  a.band_m = 1;
  a.band_t = 1;
  const int quads = m.pitch / 4;
  const int bx = quads < 64 ? quads : 64;
  const int by = vdk::kPassThreads / bx;
  const int nrb = (m.h + by - 1) / by;
  dim3 block(bx, by);
  dim3 grid((quads + bx - 1) / bx, nrb);
  // k-strided bands of row blocks, as the plain pass; auto from the step
  // whose rows y - k .. y + k span 8 MB (k >= 64 on 8192^2: JFA frame 4.31 ->
  // 4.27 ms with 2^18 seeds, 4.14 -> 4.12 with 2^14, on the GB300)
  bool band = false;
  if (band_min_k < 0) band = 2.0 * k * m.pitch * 8.0 >= 8.0 * 1024 * 1024;
  else if (band_min_k > 0) band = k >= band_min_k;
  if (band && k % by == 0 && k / by > 1) {
    a.band_m = k / by;
    a.band_t = (nrb + a.band_m - 1) / a.band_m;
    grid.y = a.band_m * a.band_t;
  }
  const bool out32 = dst32 != nullptr;
  cudaError_t e;
  if (nb == VD_NB_MOORE)
    e = metric == VD_METRIC_EUCLID ? launch_pos_t<vdk::kMoore, vdk::kEuclid>(out32, grid, block, st, pdl, a)
                                   : launch_pos_t<vdk::kMoore, vdk::kManhattan>(out32, grid, block, st, pdl, a);
  else
    e = metric == VD_METRIC_EUCLID ? launch_pos_t<vdk::kVonNeumann, vdk::kEuclid>(out32, grid, block, st, pdl, a)
                                   : launch_pos_t<vdk::kVonNeumann, vdk::kManhattan>(out32, grid, block, st, pdl, a);
  if (e != cudaSuccess) return vd_cuda_check(e, "position-map pass launch");
  return vd_cuda_check(cudaGetLastError(), "position-map pass launch");
}

}  // namespace vdi
