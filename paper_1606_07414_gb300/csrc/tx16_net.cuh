// The 44-addition fast algorithm of the 16-point approximation (Sec. 2.2):
//   T = P2 . M4 . M3 . M2 . P1 . M1
// applied to 16 values held in registers.  Works for int (exact) and float
// (each stage output is one IEEE add or subtract of two stage inputs, so the
// binary32 result is fixed by the factorisation, independent of the compiler).
//
// Stage formulas, 0-indexed:
//   M1 = [[I8, J8], [J8, -I8]]      a[i] = x[i] + x[15-i], a[8+i] = x[7-i] - x[8+i]
//   P1 (10 12 16)(11 13 15)         b[i] = a[g1[i]], g1 = 0..8,11,12,15,14,13,10,9
//   M2 = diag(B8, B8)               B8 = [[I4, J4], [J4, -I4]]
//   M3 = diag(B4, -I4, B4, -I4)     B4 = [[I2, J2], [J2, -I2]]
//   M4 = diag([[1,1,0],[1,-1,0],[0,0,-1]], I4, [[-1,0,0],[0,1,1],[0,1,-1]], -I4,
//             [[1,0],[0,-1]])
//   P2 (2 9)(3 8 16 15 5 4 12 11 7 6 10 14 13)
//                                   y[i] = e[g2[i]], g2 = 0,8,7,11,3,9,5,15,1,13,6,10,2,12,4,14
// (cycles 1-indexed as printed; (P x)_i = x_sigma(i), sigma = next element of
// the cycle -- the convention under which the product equals T).
//
// M1..M4 are symmetric, so T^t = M1 P1^t M2 M3 M4 P2^t: the inverse network
// runs the same butterflies in reverse order with the permutations scattered
// instead of gathered.
#pragma once

namespace tx16 {

// Shared butterflies of M2, M3 and M4 (the middle of the network).
template <typename V>
__device__ __forceinline__ void mid_stages(V (&b)[16], V (&e)[16]) {
  V c[16];
#pragma unroll
  for (int h = 0; h < 16; h += 8) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[h + i] = b[h + i] + b[h + 7 - i];
      c[h + 4 + i] = b[h + 3 - i] - b[h + 4 + i];
    }
  }
  V d[16];
  d[0] = c[0] + c[3];
  d[1] = c[1] + c[2];
  d[2] = c[1] - c[2];
  d[3] = c[0] - c[3];
  d[4] = -c[4];
  d[5] = -c[5];
  d[6] = -c[6];
  d[7] = -c[7];
  d[8] = c[8] + c[11];
  d[9] = c[9] + c[10];
  d[10] = c[9] - c[10];
  d[11] = c[8] - c[11];
  d[12] = -c[12];
  d[13] = -c[13];
  d[14] = -c[14];
  d[15] = -c[15];
  e[0] = d[0] + d[1];
  e[1] = d[0] - d[1];
  e[2] = -d[2];
  e[3] = d[3];
  e[4] = d[4];
  e[5] = d[5];
  e[6] = d[6];
  e[7] = -d[7];
  e[8] = d[8] + d[9];
  e[9] = d[8] - d[9];
  e[10] = -d[10];
  e[11] = -d[11];
  e[12] = -d[12];
  e[13] = -d[13];
  e[14] = d[14];
  e[15] = -d[15];
}

// x <- T x
template <typename V>
__device__ __forceinline__ void fwd16(V (&x)[16]) {
  V a[16];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    a[i] = x[i] + x[15 - i];
    a[8 + i] = x[7 - i] - x[8 + i];
  }
  V b[16] = {a[0], a[1], a[2],  a[3],  a[4],  a[5],  a[6],  a[7],
             a[8], a[11], a[12], a[15], a[14], a[13], a[10], a[9]};
  V e[16];
  mid_stages(b, e);
  x[0] = e[0];
  x[1] = e[8];
  x[2] = e[7];
  x[3] = e[11];
  x[4] = e[3];
  x[5] = e[9];
  x[6] = e[5];
  x[7] = e[15];
  x[8] = e[1];
  x[9] = e[13];
  x[10] = e[6];
  x[11] = e[10];
  x[12] = e[2];
  x[13] = e[12];
  x[14] = e[4];
  x[15] = e[14];
}

// x <- T^t x
template <typename V>
__device__ __forceinline__ void inv16(V (&x)[16]) {
  // P2^t: e[g2[i]] = x[i]
  V e[16];
  e[0] = x[0];
  e[8] = x[1];
  e[7] = x[2];
  e[11] = x[3];
  e[3] = x[4];
  e[9] = x[5];
  e[5] = x[6];
  e[15] = x[7];
  e[1] = x[8];
  e[13] = x[9];
  e[6] = x[10];
  e[10] = x[11];
  e[2] = x[12];
  e[12] = x[13];
  e[4] = x[14];
  e[14] = x[15];
  // M4, M3, M2 (each symmetric) in that order: the same butterflies as the
  // forward network's middle, applied in reverse stage order.
  V d[16];
  d[0] = e[0] + e[1];
  d[1] = e[0] - e[1];
  d[2] = -e[2];
  d[3] = e[3];
  d[4] = e[4];
  d[5] = e[5];
  d[6] = e[6];
  d[7] = -e[7];
  d[8] = e[8] + e[9];
  d[9] = e[8] - e[9];
  d[10] = -e[10];
  d[11] = -e[11];
  d[12] = -e[12];
  d[13] = -e[13];
  d[14] = e[14];
  d[15] = -e[15];
  V c[16];
  c[0] = d[0] + d[3];
  c[1] = d[1] + d[2];
  c[2] = d[1] - d[2];
  c[3] = d[0] - d[3];
  c[4] = -d[4];
  c[5] = -d[5];
  c[6] = -d[6];
  c[7] = -d[7];
  c[8] = d[8] + d[11];
  c[9] = d[9] + d[10];
  c[10] = d[9] - d[10];
  c[11] = d[8] - d[11];
  c[12] = -d[12];
  c[13] = -d[13];
  c[14] = -d[14];
  c[15] = -d[15];
  V b[16];
#pragma unroll
  for (int h = 0; h < 16; h += 8) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      b[h + i] = c[h + i] + c[h + 7 - i];
      b[h + 4 + i] = c[h + 3 - i] - c[h + 4 + i];
    }
  }
  // P1^t: a[g1[i]] = b[i]
  V a[16] = {b[0], b[1], b[2],  b[3],  b[4],  b[5],  b[6],  b[7],
             b[8], b[15], b[14], b[9], b[10], b[13], b[12], b[11]};
  // M1
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    x[i] = a[i] + a[15 - i];
    x[8 + i] = a[7 - i] - a[8 + i];
  }
}

// e(u) = log_sqrt2(4 s_u): S = (1/4) diag(1,1,2,r2,r2,1,2,2,1,2,2,r2,r2,2,2,2)
// (Sec. 2.1).  s_u s_v = sqrt2^(e(u)+e(v)) / 16, and D'_u = 16 s_u^2 = 2^e(u).
__host__ __device__ constexpr int scale_class(int u) {
  return (u == 3 || u == 4 || u == 11 || u == 12) ? 1
         : (u == 0 || u == 1 || u == 5 || u == 8) ? 0
                                                  : 2;
}

}  // namespace tx16

namespace tx16 {

// The 8-point approximation T8 from which T is built (Sec. 2.1: 14 additions):
// the halves of M2, M3 and M4 that act on the sums x_i + x_{15-i} (their
// top-left 8x8 blocks), then the outputs in frequency order, taken from the
// even rows of T:   y[k] = e[g8[k]], g8 = 0, 7, 3, 5, 1, 6, 2, 4.
//   c[i] = x[i] + x[7-i], c[4+i] = x[3-i] - x[4+i]          (B8, 8 additions)
//   d = (c0+c3, c1+c2, c1-c2, c0-c3, -c4, -c5, -c6, -c7)     (B4, -I4: 4)
//   e = (d0+d1, d0-d1, -d2, d3, d4, d5, d6, -d7)             (2)
template <typename V>
__device__ __forceinline__ void fwd8(V (&x)[8]) {
  V c[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    c[i] = x[i] + x[7 - i];
    c[4 + i] = x[3 - i] - x[4 + i];
  }
  const V d0 = c[0] + c[3], d1 = c[1] + c[2], d2 = c[1] - c[2], d3 = c[0] - c[3];
  // e0 = d0 + d1, e1 = d0 - d1, e2 = -d2, e3 = d3, e4..e6 = -c4..-c6, e7 = c7
  x[0] = d0 + d1;   // e0
  x[1] = c[7];      // e7 = -d7 = c7
  x[2] = d3;        // e3
  x[3] = -c[5];     // e5
  x[4] = d0 - d1;   // e1
  x[5] = -c[6];     // e6
  x[6] = -d2;       // e2
  x[7] = -c[4];     // e4
}

// x <- T8^t x: the same symmetric stages in reverse order, the outputs of the
// forward network scattered back (e[g8[k]] = x[k]).
template <typename V>
__device__ __forceinline__ void inv8(V (&x)[8]) {
  const V e0 = x[0], e7 = x[1], e3 = x[2], e5 = x[3], e1 = x[4], e6 = x[5], e2 = x[6], e4 = x[7];
  // M4 block: d = (e0+e1, e0-e1, -e2, e3, e4, e5, e6, -e7)
  const V d0 = e0 + e1, d1 = e0 - e1, d2 = -e2, d3 = e3;
  // B4 and -I4: c = (d0+d3, d1+d2, d1-d2, d0-d3, -e4, -e5, -e6, e7)
  V c[8];
  c[0] = d0 + d3;
  c[1] = d1 + d2;
  c[2] = d1 - d2;
  c[3] = d0 - d3;
  c[4] = -e4;
  c[5] = -e5;
  c[6] = -e6;
  c[7] = e7;
  // B8
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    x[i] = c[i] + c[7 - i];
    x[4 + i] = c[3 - i] - c[4 + i];
  }
}

}  // namespace tx16
