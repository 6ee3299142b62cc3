// predict_index.cuh -- compile-time enumerations of the factorised
// predictor (awe_predict.cu): positions of spatial and space-time modes in
// their orderings, the projection axes of the 9 flux row sets, and the same
// enumerations packed into integer constants for the strided item loops.
// Host-callable, so that tests/test_predict_indices.py can check them on the
// CPU against the host-built mode tables.
#pragma once

namespace awe {

// compile-time positions in the enumerations used by the factorised kernel
__host__ __device__ constexpr int p3idx(int b, int c) { return c * 4 - c * (c - 1) / 2 + b; }   // b+c <= 3, c outer
__host__ __device__ constexpr int p2idx(int p, int e) { return e * 3 - e * (e - 1) / 2 + p; }   // p+e <= 2, e outer
__host__ __device__ constexpr int simplex_idx(int M, int a, int b, int c) {                     // a+b+c <= M, c outer
  int idx = 0;
  for (int cc = 0; cc < c; ++cc) idx += (M - cc + 1) * (M - cc + 2) / 2;
  for (int bb = 0; bb < b; ++bb) idx += M - c - bb + 1;
  return idx + a;
}
__host__ __device__ constexpr int tri2idx(int p, int q, int r) { return simplex_idx(2, p, q, r); }
__host__ __device__ constexpr int gmidx(int a, int b, int c, int e) {                            // G-modes, e outer
  return (e == 0 ? 0 : e == 1 ? 10 : 14) + simplex_idx(2 - e, a, b, c);
}
// the (p, q, r) of tri2 index t, as compile-time functions
__host__ __device__ constexpr int tri2_p(int t) {
  for (int r = 0; r <= 2; ++r)
    for (int q = 0; q <= 2 - r; ++q)
      for (int p = 0; p <= 2 - r - q; ++p)
        if (tri2idx(p, q, r) == t) return p;
  return -1;
}
__host__ __device__ constexpr int tri2_q(int t) {
  for (int r = 0; r <= 2; ++r)
    for (int q = 0; q <= 2 - r; ++q)
      for (int p = 0; p <= 2 - r - q; ++p)
        if (tri2idx(p, q, r) == t) return q;
  return -1;
}
__host__ __device__ constexpr int tri2_r(int t) {
  for (int r = 0; r <= 2; ++r)
    for (int q = 0; q <= 2 - r; ++q)
      for (int p = 0; p <= 2 - r - q; ++p)
        if (tri2idx(p, q, r) == t) return r;
  return -1;
}
__host__ __device__ constexpr int pair2_p(int pe) { return pe < 3 ? pe : pe < 5 ? pe - 3 : 0; }
__host__ __device__ constexpr int pair2_e(int pe) { return pe < 3 ? 0 : pe < 5 ? 1 : 2; }

// The same enumerations decoded with integer arithmetic on packed constants
// (2 or 4 bits per entry), for the strided item loops: an index table in
// shared memory would put a dependent load in front of every operand load.
__host__ __device__ constexpr unsigned long long pack_bits(int n, int bits, int which) {
  unsigned long long k = 0;
  for (int i = 0; i < n; ++i) {
    int v = 0;
    switch (which) {
      case 0: v = tri2_p(i); break;
      case 1: v = tri2_q(i); break;
      case 2: v = tri2_r(i); break;
      default: v = 0;
    }
    k |= (unsigned long long)v << (bits * i);
  }
  return k;
}
// projection axes of the 9 flux row sets and the (d, v') combinations (fact_project)
__host__ __device__ constexpr int p1c1_of(int r) { return r == 2 || r == 4 || r == 8 ? 1 : r == 5 ? 0 : 2; }
__host__ __device__ constexpr int p2row_of(int dv) {
  return dv % 4 == 3 ? 6 + dv / 4
       : dv % 4 == dv / 4 ? dv / 4
       : 3 + dv % 4 + dv / 4 - 1;
}
__host__ __device__ constexpr bool p2lo_of(int dv) {   // d is the lower of the two axes P1 leaves
  return dv / 4 == (p1c1_of(p2row_of(dv)) == 0 ? 1 : 0);
}
__host__ __device__ constexpr bool p2swap_of(int dv) {  // the P2 axis is above the P1 axis
  return (p2lo_of(dv) ? (p1c1_of(p2row_of(dv)) == 2 ? 1 : 2) : (p1c1_of(p2row_of(dv)) == 0 ? 1 : 0)) >
         p1c1_of(p2row_of(dv));
}
__host__ __device__ constexpr unsigned long long pack_proj(int which) {
  unsigned long long k = 0;
  for (int i = 0; i < 12; ++i) {
    const unsigned long long v = which == 0 ? (i < 9 ? p1c1_of(i) : 0)
                               : which == 1 ? p2row_of(i)
                               : which == 2 ? p2lo_of(i) : p2swap_of(i);
    k |= v << (4 * i);
  }
  return k;
}
constexpr unsigned long long kTri2P = pack_bits(10, 2, 0), kTri2Q = pack_bits(10, 2, 1), kTri2R = pack_bits(10, 2, 2);
constexpr unsigned long long kP1C1 = pack_proj(0), kP2Row = pack_proj(1), kP2Lo = pack_proj(2), kP2Swap = pack_proj(3);
__host__ __device__ __forceinline__ int unpack(unsigned long long k, int bits, int i) {
  return (int)((k >> (bits * i)) & ((1ull << bits) - 1));
}
// index of (a, b, c), a + b + c <= 2, c outermost (= tri2idx)
__host__ __device__ __forceinline__ int tri2_fast(int a, int b, int c) {
  return (c == 0 ? 0 : c == 1 ? 6 : 9) + b * (3 - c) - (b * (b - 1)) / 2 + a;
}
// G-mode (a, b, c, e) of degree <= 2 (= gmidx)
__host__ __device__ __forceinline__ int gm_fast(int a, int b, int c, int e) {
  return e == 0 ? tri2_fast(a, b, c) : e == 1 ? 10 + (c ? 3 : b ? 2 : a) : 14;
}
// exponents of G-mode i (15 modes, e outermost)
__host__ __device__ constexpr unsigned long long pack_gm(int k) {
  unsigned long long r = 0;
  int i = 0;
  for (int e = 0; e <= 2; ++e)
    for (int c = 0; c <= 2 - e; ++c)
      for (int b = 0; b <= 2 - e - c; ++b)
        for (int a = 0; a <= 2 - e - b - c; ++a) {
          const int v = k == 0 ? a : k == 1 ? b : k == 2 ? c : e;
          r |= (unsigned long long)v << (2 * i++);
        }
  return r;
}
constexpr unsigned long long kGmA = pack_gm(0), kGmB = pack_gm(1), kGmC = pack_gm(2), kGmE = pack_gm(3);

}  // namespace awe
