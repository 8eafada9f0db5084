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
#ifdef __CUDACC__
#include <cuda_runtime.h>
#endif

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

#ifdef __CUDACC__
// FP32 pair (hi, lo) of an FP64 value q: hi is q truncated to 24 significant
// bits, lo = q - hi (exact in FP64) rounded to FP32, so hi + lo equals q to
// about 2^-47 relative.  Built from the bits of q with integer operations,
// off the FP64 pipe (1/64 of the FP32 rate on this part; the conversions of
// the plain form (float)q, (float)(q - (double)hi) ran on it).  Exponents
// outside the range where hi and lo are normal FP32 numbers take that plain
// form; zero (and FP64 subnormals) give (0, 0) with the sign of q.
__device__ __forceinline__ void split_hilo(double q, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(q);
  const unsigned hw = (unsigned)(b >> 32);
  const int e = (int)((hw >> 20) & 0x7ffu);
  const unsigned sign = hw & 0x80000000u;
  if (e >= 950 && e <= 1150) {
    // hi: sign, exponent rebased from 1023 to 127, top 23 mantissa bits
    hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
    // lo: the 29 dropped mantissa bits times 2^(e - 1075), rounded once
    const unsigned rem = (unsigned)(b & 0x1fffffffu);
    const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);
    lo = __uint_as_float(__float_as_uint(__uint2float_rn(rem) * scale) | sign);
  } else if (e == 0) {
    hi = __uint_as_float(sign);
    lo = hi;
  } else {
    hi = (float)q;
    lo = (float)(q - (double)hi);
  }
}

#endif

}  // namespace cw
