// Device layouts of the per-cell reconstruction data, shared by the kernels
// that write them (least-squares setup, moving-mesh rebuild) and the
// reconstruction kernel that reads them.
//
//   R_i (pseudo-inverse of Eq. CWENO:Popt), entry (stencil neighbour r,
//   coefficient k) flattened as e = r (Mc - 1) + k and stored in 16-byte
//   vectors of VW = 16 / sizeof(T) entries: vector g = e / VW of cell i at
//   [(g N + i) VW + e mod VW].  One warp reading vector g of 32 consecutive
//   cells reads 512 contiguous bytes; four neighbours' entries form whole
//   vectors, so the kernel loads them as 128-bit values.
//
//   Central stencil ids, four per 16-byte vector: neighbour r of cell i at
//   [((r / 4) N + i) 4 + r mod 4], the unused slots of the last vector hold i.
//
//   FP32 pair copy of the cell averages (FP32-mixed mode), interleaved per
//   cell: (hi, lo) of variable v of cell i at [(i NVP + v) 2], NVP = nv
//   rounded up to even, so one cell's pairs are NVP / 2 16-byte vectors.
#pragma once
#include <cstdint>

namespace cw {

template <typename T>
__host__ __device__ constexpr int vec_width() {
  return 16 / (int)sizeof(T);
}
__host__ __device__ constexpr int r_vectors(int ne1, int mc1, int vw) { return (ne1 * mc1 + vw - 1) / vw; }
template <typename T>
__host__ __device__ inline int64_t r_index(int r, int k, int mc1, int64_t i, int64_t N) {
  constexpr int vw = vec_width<T>();
  const int e = r * mc1 + k;
  return ((int64_t)(e / vw) * N + i) * vw + e % vw;
}
__host__ __device__ constexpr int sten_vectors(int ne1) { return (ne1 + 3) / 4; }
__host__ __device__ constexpr int pair_vars(int nv) { return (nv + 1) & ~1; }

}  // namespace cw
