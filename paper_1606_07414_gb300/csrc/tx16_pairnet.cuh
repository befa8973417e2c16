// GENERATED by gen_networks.py -- do not edit.  The 44-addition network of
// T = P2 M4 M3 M2 P1 M1 (Sec. 2.2) on float2 pairs, negations folded into the
// additions and pruned to the zonal extents used by the fused codec.
#pragma once
#include <cuda_runtime.h>
namespace tx16 {
namespace pairnet {
__device__ __forceinline__ float2 pm1() { return make_float2(-1.f, -1.f); }
__device__ __forceinline__ float2 pbias() { return make_float2(-16777216.f, -16777216.f); }  // -2^24
// a - b and RD(a - b) per lane: a packed addition of the negated operand
// (one rounding; the negation folds into the instruction)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 sub2_rd(float2 a, float2 b) { return __fadd2_rd(a, make_float2(-b.x, -b.y)); }
// sign of output i encoded as bit masks (negative / known zero)
__host__ __device__ constexpr int sign_of(unsigned neg, unsigned zero, int i) {
  return ((zero >> i) & 1u) ? 0 : (((neg >> i) & 1u) ? -1 : 1);
}

// forward row pass, outputs v < 4: y[v] = sign[v] * (T x)[v]; 16 pair additions after M1
struct FwdRow4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xfff0u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {
    const float2 a0 = __fadd2_rn(__fadd2_rn(X[0], pbias()), X[15]);
    const float2 a15 = sub2(X[0], X[15]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = sub2(X[1], X[14]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = sub2(X[2], X[13]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = sub2(X[3], X[12]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = sub2(X[4], X[11]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = sub2(X[5], X[10]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = sub2(X[6], X[9]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = sub2(X[7], X[8]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = sub2(a0, a7);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    y[0] = t40;
    y[1] = t42;
    y[2] = t23;
    y[3] = t39;
    y[4] = make_float2(0.f, 0.f);
    y[5] = make_float2(0.f, 0.f);
    y[6] = make_float2(0.f, 0.f);
    y[7] = make_float2(0.f, 0.f);
    y[8] = make_float2(0.f, 0.f);
    y[9] = make_float2(0.f, 0.f);
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward row pass, outputs v < 6: y[v] = sign[v] * (T x)[v]; 18 pair additions after M1
struct FwdRow6 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xffc0u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {
    const float2 a0 = __fadd2_rn(__fadd2_rn(X[0], pbias()), X[15]);
    const float2 a15 = sub2(X[0], X[15]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = sub2(X[1], X[14]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = sub2(X[2], X[13]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = sub2(X[3], X[12]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = sub2(X[4], X[11]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = sub2(X[5], X[10]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = sub2(X[6], X[9]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = sub2(X[7], X[8]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = sub2(a0, a7);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    y[0] = t40;
    y[1] = t42;
    y[2] = t23;
    y[3] = t39;
    y[4] = t35;
    y[5] = t43;
    y[6] = make_float2(0.f, 0.f);
    y[7] = make_float2(0.f, 0.f);
    y[8] = make_float2(0.f, 0.f);
    y[9] = make_float2(0.f, 0.f);
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward row pass, outputs v < 8: y[v] = sign[v] * (T x)[v]; 20 pair additions after M1
struct FwdRow8 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {
    const float2 a0 = __fadd2_rn(__fadd2_rn(X[0], pbias()), X[15]);
    const float2 a15 = sub2(X[0], X[15]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = sub2(X[1], X[14]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = sub2(X[2], X[13]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = sub2(X[3], X[12]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = sub2(X[4], X[11]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = sub2(X[5], X[10]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = sub2(X[6], X[9]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = sub2(X[7], X[8]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t19 = sub2(a2, a5);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = sub2(a0, a7);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t31 = sub2(a8, a9);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    y[0] = t40;
    y[1] = t42;
    y[2] = t23;
    y[3] = t39;
    y[4] = t35;
    y[5] = t43;
    y[6] = t19;
    y[7] = t31;
    y[8] = make_float2(0.f, 0.f);
    y[9] = make_float2(0.f, 0.f);
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward row pass, outputs v < 10: y[v] = sign[v] * (T x)[v]; 22 pair additions after M1
struct FwdRow10 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xfc00u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {
    const float2 a0 = __fadd2_rn(__fadd2_rn(X[0], pbias()), X[15]);
    const float2 a15 = sub2(X[0], X[15]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = sub2(X[1], X[14]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = sub2(X[2], X[13]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = sub2(X[3], X[12]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = sub2(X[4], X[11]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = sub2(X[5], X[10]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = sub2(X[6], X[9]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = sub2(X[7], X[8]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t19 = sub2(a2, a5);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = sub2(a0, a7);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t27 = sub2(a12, a13);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t31 = sub2(a8, a9);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    y[0] = t40;
    y[1] = t42;
    y[2] = t23;
    y[3] = t39;
    y[4] = t35;
    y[5] = t43;
    y[6] = t19;
    y[7] = t31;
    y[8] = t41;
    y[9] = t27;
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward row pass, outputs v < 16: y[v] = sign[v] * (T x)[v]; 28 pair additions after M1
struct FwdRow16 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0xdc48u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {
    const float2 a0 = __fadd2_rn(__fadd2_rn(X[0], pbias()), X[15]);
    const float2 a15 = sub2(X[0], X[15]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = sub2(X[1], X[14]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = sub2(X[2], X[13]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = sub2(X[3], X[12]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = sub2(X[4], X[11]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = sub2(X[5], X[10]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = sub2(X[6], X[9]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = sub2(X[7], X[8]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t17 = sub2(a3, a4);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t19 = sub2(a2, a5);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t21 = sub2(a1, a6);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = sub2(a0, a7);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t25 = sub2(a15, a14);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t27 = sub2(a12, a13);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t29 = sub2(a11, a10);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t31 = sub2(a8, a9);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t34 = sub2(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = sub2(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    y[0] = t40;
    y[1] = t42;
    y[2] = t23;
    y[3] = t39;
    y[4] = t35;
    y[5] = t43;
    y[6] = t19;
    y[7] = t31;
    y[8] = t41;
    y[9] = t27;
    y[10] = t21;
    y[11] = t38;
    y[12] = t34;
    y[13] = t25;
    y[14] = t17;
    y[15] = t29;
  }
};

// forward column pass, outputs u < 3: y[u] = sign[u] * (T x)[u]; 31 pair additions
struct FwdCol3 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfff8u, i); }
  __device__ static __forceinline__ void run(const float2 (&x)[16], float2 (&y)[16]) {
    const float2 t16 = __fadd2_rn(x[0], x[15]);
    const float2 t17 = sub2(x[7], x[8]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = sub2(x[6], x[9]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = sub2(x[5], x[10]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = sub2(x[4], x[11]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = sub2(x[3], x[12]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = sub2(x[2], x[13]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = sub2(x[1], x[14]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = sub2(x[0], x[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    y[0] = t56;
    y[1] = t58;
    y[2] = t39;
    y[3] = make_float2(0.f, 0.f);
    y[4] = make_float2(0.f, 0.f);
    y[5] = make_float2(0.f, 0.f);
    y[6] = make_float2(0.f, 0.f);
    y[7] = make_float2(0.f, 0.f);
    y[8] = make_float2(0.f, 0.f);
    y[9] = make_float2(0.f, 0.f);
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward column pass, outputs u < 5: y[u] = sign[u] * (T x)[u]; 33 pair additions
struct FwdCol5 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xffe0u, i); }
  __device__ static __forceinline__ void run(const float2 (&x)[16], float2 (&y)[16]) {
    const float2 t16 = __fadd2_rn(x[0], x[15]);
    const float2 t17 = sub2(x[7], x[8]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = sub2(x[6], x[9]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = sub2(x[5], x[10]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = sub2(x[4], x[11]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = sub2(x[3], x[12]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = sub2(x[2], x[13]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = sub2(x[1], x[14]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = sub2(x[0], x[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    y[0] = t56;
    y[1] = t58;
    y[2] = t39;
    y[3] = t55;
    y[4] = t51;
    y[5] = make_float2(0.f, 0.f);
    y[6] = make_float2(0.f, 0.f);
    y[7] = make_float2(0.f, 0.f);
    y[8] = make_float2(0.f, 0.f);
    y[9] = make_float2(0.f, 0.f);
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward column pass, outputs u < 7: y[u] = sign[u] * (T x)[u]; 35 pair additions
struct FwdCol7 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xff80u, i); }
  __device__ static __forceinline__ void run(const float2 (&x)[16], float2 (&y)[16]) {
    const float2 t16 = __fadd2_rn(x[0], x[15]);
    const float2 t17 = sub2(x[7], x[8]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = sub2(x[6], x[9]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = sub2(x[5], x[10]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = sub2(x[4], x[11]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = sub2(x[3], x[12]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = sub2(x[2], x[13]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = sub2(x[1], x[14]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = sub2(x[0], x[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = sub2(t20, t26);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    y[0] = t56;
    y[1] = t58;
    y[2] = t39;
    y[3] = t55;
    y[4] = t51;
    y[5] = t59;
    y[6] = t35;
    y[7] = make_float2(0.f, 0.f);
    y[8] = make_float2(0.f, 0.f);
    y[9] = make_float2(0.f, 0.f);
    y[10] = make_float2(0.f, 0.f);
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward column pass, outputs u < 11: y[u] = sign[u] * (T x)[u]; 39 pair additions
struct FwdCol11 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0448u, 0xf800u, i); }
  __device__ static __forceinline__ void run(const float2 (&x)[16], float2 (&y)[16]) {
    const float2 t16 = __fadd2_rn(x[0], x[15]);
    const float2 t17 = sub2(x[7], x[8]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = sub2(x[6], x[9]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = sub2(x[5], x[10]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = sub2(x[4], x[11]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = sub2(x[3], x[12]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = sub2(x[2], x[13]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = sub2(x[1], x[14]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = sub2(x[0], x[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = sub2(t20, t26);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t37 = sub2(t18, t28);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t43 = sub2(t25, t27);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = sub2(t17, t19);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t57 = sub2(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    y[0] = t56;
    y[1] = t58;
    y[2] = t39;
    y[3] = t55;
    y[4] = t51;
    y[5] = t59;
    y[6] = t35;
    y[7] = t47;
    y[8] = t57;
    y[9] = t43;
    y[10] = t37;
    y[11] = make_float2(0.f, 0.f);
    y[12] = make_float2(0.f, 0.f);
    y[13] = make_float2(0.f, 0.f);
    y[14] = make_float2(0.f, 0.f);
    y[15] = make_float2(0.f, 0.f);
  }
};

// forward column pass, outputs u < 16: y[u] = sign[u] * (T x)[u]; 44 pair additions
struct FwdCol16 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0xdc48u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&x)[16], float2 (&y)[16]) {
    const float2 t16 = __fadd2_rn(x[0], x[15]);
    const float2 t17 = sub2(x[7], x[8]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = sub2(x[6], x[9]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = sub2(x[5], x[10]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = sub2(x[4], x[11]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = sub2(x[3], x[12]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = sub2(x[2], x[13]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = sub2(x[1], x[14]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = sub2(x[0], x[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t33 = sub2(t22, t24);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = sub2(t20, t26);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t37 = sub2(t18, t28);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t41 = sub2(t31, t29);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t43 = sub2(t25, t27);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t45 = sub2(t23, t21);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = sub2(t17, t19);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t50 = sub2(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t54 = sub2(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t57 = sub2(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    y[0] = t56;
    y[1] = t58;
    y[2] = t39;
    y[3] = t55;
    y[4] = t51;
    y[5] = t59;
    y[6] = t35;
    y[7] = t47;
    y[8] = t57;
    y[9] = t43;
    y[10] = t37;
    y[11] = t54;
    y[12] = t50;
    y[13] = t41;
    y[14] = t33;
    y[15] = t45;
  }
};

// inverse column pass, inputs u < 3 (node values, signs of the forward column
// pass), outputs z[i] = (T^t w)[i] materialised; 18 pair additions
struct InvCol3 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t3 = __fadd2_rn(w[0], w[2]);
    const float2 t4 = sub2(w[0], w[2]);
    const float2 t5 = __fadd2_rn(t3, w[1]);
    const float2 t6 = sub2(t4, w[1]);
    const float2 t7 = __fadd2_rn(w[0], w[1]);
    const float2 t8 = sub2(w[0], w[1]);
    const float2 t9 = __fadd2_rn(w[0], w[1]);
    const float2 t10 = sub2(w[0], w[1]);
    const float2 t11 = __fadd2_rn(w[0], w[1]);
    const float2 t12 = sub2(w[0], w[1]);
    const float2 t13 = __fadd2_rn(w[0], w[1]);
    const float2 t14 = sub2(w[0], w[1]);
    const float2 t15 = __fadd2_rn(w[0], w[1]);
    const float2 t16 = sub2(w[0], w[1]);
    const float2 t17 = __fadd2_rn(w[0], w[1]);
    const float2 t18 = sub2(w[0], w[1]);
    const float2 t19 = __fadd2_rn(t4, w[1]);
    const float2 t20 = sub2(t3, w[1]);
    z[0] = t5;
    z[1] = t7;
    z[2] = t9;
    z[3] = t11;
    z[4] = t13;
    z[5] = t15;
    z[6] = t17;
    z[7] = t19;
    z[8] = t6;
    z[9] = t8;
    z[10] = t10;
    z[11] = t12;
    z[12] = t14;
    z[13] = t16;
    z[14] = t18;
    z[15] = t20;
  }
};

// inverse column pass, inputs u < 5 (node values, signs of the forward column
// pass), outputs z[i] = (T^t w)[i] materialised; 22 pair additions
struct InvCol5 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t5 = __fadd2_rn(w[0], w[4]);
    const float2 t6 = sub2(w[0], w[4]);
    const float2 t7 = __fadd2_rn(w[1], w[3]);
    const float2 t8 = sub2(w[1], w[3]);
    const float2 t9 = __fadd2_rn(t5, w[2]);
    const float2 t10 = sub2(t5, w[2]);
    const float2 t11 = __fadd2_rn(t9, t8);
    const float2 t12 = sub2(t10, t7);
    const float2 t13 = __fadd2_rn(w[0], t8);
    const float2 t14 = sub2(w[0], t7);
    const float2 t15 = __fadd2_rn(w[0], w[1]);
    const float2 t16 = sub2(w[0], w[1]);
    const float2 t17 = __fadd2_rn(t6, w[1]);
    const float2 t18 = sub2(t6, w[1]);
    const float2 t19 = __fadd2_rn(t6, w[1]);
    const float2 t20 = sub2(t6, w[1]);
    const float2 t21 = __fadd2_rn(w[0], w[1]);
    const float2 t22 = sub2(w[0], w[1]);
    const float2 t23 = __fadd2_rn(w[0], t7);
    const float2 t24 = sub2(w[0], t8);
    const float2 t25 = __fadd2_rn(t10, t7);
    const float2 t26 = sub2(t9, t8);
    z[0] = t11;
    z[1] = t13;
    z[2] = t15;
    z[3] = t17;
    z[4] = t19;
    z[5] = t21;
    z[6] = t23;
    z[7] = t25;
    z[8] = t12;
    z[9] = t14;
    z[10] = t16;
    z[11] = t18;
    z[12] = t20;
    z[13] = t22;
    z[14] = t24;
    z[15] = t26;
  }
};

// inverse column pass, inputs u < 7 (node values, signs of the forward column
// pass), outputs z[i] = (T^t w)[i] materialised; 26 pair additions
struct InvCol7 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t7 = __fadd2_rn(w[1], w[5]);
    const float2 t8 = sub2(w[1], w[5]);
    const float2 t9 = __fadd2_rn(w[0], w[4]);
    const float2 t10 = sub2(w[0], w[4]);
    const float2 t11 = __fadd2_rn(t7, w[3]);
    const float2 t12 = sub2(t7, w[3]);
    const float2 t13 = __fadd2_rn(t9, w[2]);
    const float2 t14 = sub2(w[0], w[6]);
    const float2 t15 = __fadd2_rn(w[0], w[6]);
    const float2 t16 = sub2(t9, w[2]);
    const float2 t17 = __fadd2_rn(t13, t12);
    const float2 t18 = sub2(t16, t11);
    const float2 t19 = __fadd2_rn(w[0], t12);
    const float2 t20 = sub2(w[0], t11);
    const float2 t21 = __fadd2_rn(t15, t8);
    const float2 t22 = sub2(t14, t8);
    const float2 t23 = __fadd2_rn(t10, t8);
    const float2 t24 = sub2(t10, t8);
    const float2 t25 = __fadd2_rn(t10, t8);
    const float2 t26 = sub2(t10, t8);
    const float2 t27 = __fadd2_rn(t14, t8);
    const float2 t28 = sub2(t15, t8);
    const float2 t29 = __fadd2_rn(w[0], t11);
    const float2 t30 = sub2(w[0], t12);
    const float2 t31 = __fadd2_rn(t16, t11);
    const float2 t32 = sub2(t13, t12);
    z[0] = t17;
    z[1] = t19;
    z[2] = t21;
    z[3] = t23;
    z[4] = t25;
    z[5] = t27;
    z[6] = t29;
    z[7] = t31;
    z[8] = t18;
    z[9] = t20;
    z[10] = t22;
    z[11] = t24;
    z[12] = t26;
    z[13] = t28;
    z[14] = t30;
    z[15] = t32;
  }
};

// inverse column pass, inputs u < 11 (node values, signs of the forward column
// pass), outputs z[i] = (T^t w)[i] materialised; 34 pair additions
struct InvCol11 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t11 = __fadd2_rn(w[0], w[8]);
    const float2 t12 = sub2(w[0], w[8]);
    const float2 t13 = __fadd2_rn(w[1], w[5]);
    const float2 t14 = sub2(w[1], w[5]);
    const float2 t15 = __fadd2_rn(t11, w[4]);
    const float2 t16 = sub2(t11, w[4]);
    const float2 t17 = __fadd2_rn(t13, w[3]);
    const float2 t18 = sub2(t13, w[3]);
    const float2 t19 = __fadd2_rn(t15, w[2]);
    const float2 t20 = __fadd2_rn(t12, w[10]);
    const float2 t21 = sub2(t12, w[6]);
    const float2 t22 = __fadd2_rn(t12, w[6]);
    const float2 t23 = sub2(t12, w[10]);
    const float2 t24 = sub2(t15, w[2]);
    const float2 t25 = __fadd2_rn(t17, w[7]);
    const float2 t26 = sub2(t14, w[9]);
    const float2 t27 = __fadd2_rn(t14, w[9]);
    const float2 t28 = sub2(t17, w[7]);
    const float2 t29 = __fadd2_rn(t19, t18);
    const float2 t30 = sub2(t24, t25);
    const float2 t31 = __fadd2_rn(t20, t18);
    const float2 t32 = sub2(t23, t28);
    const float2 t33 = __fadd2_rn(t22, t26);
    const float2 t34 = sub2(t21, t14);
    const float2 t35 = __fadd2_rn(t16, t27);
    const float2 t36 = sub2(t16, t14);
    const float2 t37 = __fadd2_rn(t16, t14);
    const float2 t38 = sub2(t16, t27);
    const float2 t39 = __fadd2_rn(t21, t14);
    const float2 t40 = sub2(t22, t26);
    const float2 t41 = __fadd2_rn(t23, t28);
    const float2 t42 = sub2(t20, t18);
    const float2 t43 = __fadd2_rn(t24, t25);
    const float2 t44 = sub2(t19, t18);
    z[0] = t29;
    z[1] = t31;
    z[2] = t33;
    z[3] = t35;
    z[4] = t37;
    z[5] = t39;
    z[6] = t41;
    z[7] = t43;
    z[8] = t30;
    z[9] = t32;
    z[10] = t34;
    z[11] = t36;
    z[12] = t38;
    z[13] = t40;
    z[14] = t42;
    z[15] = t44;
  }
};

// inverse column pass, inputs u < 16 (node values, signs of the forward column
// pass), outputs z[i] = (T^t w)[i] materialised; 44 pair additions
struct InvCol16 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t16 = __fadd2_rn(w[0], w[8]);
    const float2 t17 = sub2(w[0], w[8]);
    const float2 t18 = __fadd2_rn(w[1], w[5]);
    const float2 t19 = sub2(w[1], w[5]);
    const float2 t20 = __fadd2_rn(t16, w[4]);
    const float2 t21 = __fadd2_rn(t17, w[12]);
    const float2 t22 = sub2(t17, w[12]);
    const float2 t23 = sub2(t16, w[4]);
    const float2 t24 = __fadd2_rn(t18, w[3]);
    const float2 t25 = __fadd2_rn(t19, w[11]);
    const float2 t26 = sub2(t19, w[11]);
    const float2 t27 = sub2(t18, w[3]);
    const float2 t28 = __fadd2_rn(t20, w[2]);
    const float2 t29 = sub2(t23, w[14]);
    const float2 t30 = __fadd2_rn(t21, w[10]);
    const float2 t31 = sub2(t22, w[6]);
    const float2 t32 = __fadd2_rn(t22, w[6]);
    const float2 t33 = sub2(t21, w[10]);
    const float2 t34 = __fadd2_rn(t23, w[14]);
    const float2 t35 = sub2(t20, w[2]);
    const float2 t36 = __fadd2_rn(t24, w[7]);
    const float2 t37 = sub2(t27, w[13]);
    const float2 t38 = __fadd2_rn(t25, w[15]);
    const float2 t39 = sub2(t26, w[9]);
    const float2 t40 = __fadd2_rn(t26, w[9]);
    const float2 t41 = sub2(t25, w[15]);
    const float2 t42 = __fadd2_rn(t27, w[13]);
    const float2 t43 = sub2(t24, w[7]);
    const float2 t44 = __fadd2_rn(t28, t42);
    const float2 t45 = sub2(t35, t36);
    const float2 t46 = __fadd2_rn(t30, t37);
    const float2 t47 = sub2(t33, t43);
    const float2 t48 = __fadd2_rn(t32, t39);
    const float2 t49 = sub2(t31, t41);
    const float2 t50 = __fadd2_rn(t34, t40);
    const float2 t51 = sub2(t29, t38);
    const float2 t52 = __fadd2_rn(t29, t38);
    const float2 t53 = sub2(t34, t40);
    const float2 t54 = __fadd2_rn(t31, t41);
    const float2 t55 = sub2(t32, t39);
    const float2 t56 = __fadd2_rn(t33, t43);
    const float2 t57 = sub2(t30, t37);
    const float2 t58 = __fadd2_rn(t35, t36);
    const float2 t59 = sub2(t28, t42);
    z[0] = t44;
    z[1] = t46;
    z[2] = t48;
    z[3] = t50;
    z[4] = t52;
    z[5] = t54;
    z[6] = t56;
    z[7] = t58;
    z[8] = t45;
    z[9] = t47;
    z[10] = t49;
    z[11] = t51;
    z[12] = t53;
    z[13] = t55;
    z[14] = t57;
    z[15] = t59;
  }
};

// inverse row pass, inputs v < 4: z[j] = sign[j] * (T^t w)[j]; 20 pair additions
struct InvRow4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t4 = sub2(w[1], w[3]);
    const float2 t5 = __fadd2_rn(w[1], w[3]);
    const float2 t6 = __fadd2_rn(w[0], w[2]);
    const float2 t7 = sub2(w[0], w[2]);
    const float2 t8 = __fadd2_rn(t6, t5);
    const float2 t9 = sub2(t7, t4);
    const float2 t10 = __fadd2_rn(w[0], t5);
    const float2 t11 = sub2(w[0], t4);
    const float2 t12 = __fadd2_rn(w[0], w[1]);
    const float2 t13 = sub2(w[0], w[1]);
    const float2 t14 = __fadd2_rn(w[0], w[1]);
    const float2 t15 = sub2(w[0], w[1]);
    const float2 t16 = __fadd2_rn(w[0], w[1]);
    const float2 t17 = sub2(w[0], w[1]);
    const float2 t18 = __fadd2_rn(w[0], w[1]);
    const float2 t19 = sub2(w[0], w[1]);
    const float2 t20 = __fadd2_rn(w[0], t4);
    const float2 t21 = sub2(w[0], t5);
    const float2 t22 = __fadd2_rn(t7, t4);
    const float2 t23 = sub2(t6, t5);
    z[0] = t8;
    z[1] = t10;
    z[2] = t12;
    z[3] = t14;
    z[4] = t16;
    z[5] = t18;
    z[6] = t20;
    z[7] = t22;
    z[8] = t9;
    z[9] = t11;
    z[10] = t13;
    z[11] = t15;
    z[12] = t17;
    z[13] = t19;
    z[14] = t21;
    z[15] = t23;
  }
};

// inverse row pass, inputs v < 6: z[j] = sign[j] * (T^t w)[j]; 24 pair additions
struct InvRow6 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t6 = __fadd2_rn(w[1], w[5]);
    const float2 t7 = sub2(w[1], w[5]);
    const float2 t8 = __fadd2_rn(w[0], w[4]);
    const float2 t9 = sub2(w[0], w[4]);
    const float2 t10 = sub2(t6, w[3]);
    const float2 t11 = __fadd2_rn(t6, w[3]);
    const float2 t12 = __fadd2_rn(t8, w[2]);
    const float2 t13 = sub2(t8, w[2]);
    const float2 t14 = __fadd2_rn(t12, t11);
    const float2 t15 = sub2(t13, t10);
    const float2 t16 = __fadd2_rn(w[0], t11);
    const float2 t17 = sub2(w[0], t10);
    const float2 t18 = __fadd2_rn(w[0], t7);
    const float2 t19 = sub2(w[0], t7);
    const float2 t20 = __fadd2_rn(t9, t7);
    const float2 t21 = sub2(t9, t7);
    const float2 t22 = __fadd2_rn(t9, t7);
    const float2 t23 = sub2(t9, t7);
    const float2 t24 = __fadd2_rn(w[0], t7);
    const float2 t25 = sub2(w[0], t7);
    const float2 t26 = __fadd2_rn(w[0], t10);
    const float2 t27 = sub2(w[0], t11);
    const float2 t28 = __fadd2_rn(t13, t10);
    const float2 t29 = sub2(t12, t11);
    z[0] = t14;
    z[1] = t16;
    z[2] = t18;
    z[3] = t20;
    z[4] = t22;
    z[5] = t24;
    z[6] = t26;
    z[7] = t28;
    z[8] = t15;
    z[9] = t17;
    z[10] = t19;
    z[11] = t21;
    z[12] = t23;
    z[13] = t25;
    z[14] = t27;
    z[15] = t29;
  }
};

// inverse row pass, inputs v < 8: z[j] = sign[j] * (T^t w)[j]; 28 pair additions
struct InvRow8 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t8 = __fadd2_rn(w[1], w[5]);
    const float2 t9 = sub2(w[1], w[5]);
    const float2 t10 = __fadd2_rn(w[0], w[4]);
    const float2 t11 = sub2(w[0], w[4]);
    const float2 t12 = sub2(t8, w[3]);
    const float2 t13 = __fadd2_rn(t8, w[3]);
    const float2 t14 = __fadd2_rn(t10, w[2]);
    const float2 t15 = __fadd2_rn(w[0], w[6]);
    const float2 t16 = sub2(w[0], w[6]);
    const float2 t17 = sub2(t10, w[2]);
    const float2 t18 = __fadd2_rn(t12, w[7]);
    const float2 t19 = sub2(t12, w[7]);
    const float2 t20 = __fadd2_rn(t14, t13);
    const float2 t21 = sub2(t17, t18);
    const float2 t22 = __fadd2_rn(w[0], t13);
    const float2 t23 = sub2(w[0], t19);
    const float2 t24 = __fadd2_rn(t16, t9);
    const float2 t25 = sub2(t15, t9);
    const float2 t26 = __fadd2_rn(t11, t9);
    const float2 t27 = sub2(t11, t9);
    const float2 t28 = __fadd2_rn(t11, t9);
    const float2 t29 = sub2(t11, t9);
    const float2 t30 = __fadd2_rn(t15, t9);
    const float2 t31 = sub2(t16, t9);
    const float2 t32 = __fadd2_rn(w[0], t19);
    const float2 t33 = sub2(w[0], t13);
    const float2 t34 = __fadd2_rn(t17, t18);
    const float2 t35 = sub2(t14, t13);
    z[0] = t20;
    z[1] = t22;
    z[2] = t24;
    z[3] = t26;
    z[4] = t28;
    z[5] = t30;
    z[6] = t32;
    z[7] = t34;
    z[8] = t21;
    z[9] = t23;
    z[10] = t25;
    z[11] = t27;
    z[12] = t29;
    z[13] = t31;
    z[14] = t33;
    z[15] = t35;
  }
};

// inverse row pass, inputs v < 10: z[j] = sign[j] * (T^t w)[j]; 32 pair additions
struct InvRow10 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t10 = __fadd2_rn(w[0], w[8]);
    const float2 t11 = sub2(w[0], w[8]);
    const float2 t12 = __fadd2_rn(w[1], w[5]);
    const float2 t13 = sub2(w[1], w[5]);
    const float2 t14 = __fadd2_rn(t10, w[4]);
    const float2 t15 = sub2(t10, w[4]);
    const float2 t16 = sub2(t12, w[3]);
    const float2 t17 = __fadd2_rn(t12, w[3]);
    const float2 t18 = __fadd2_rn(t14, w[2]);
    const float2 t19 = __fadd2_rn(t11, w[6]);
    const float2 t20 = sub2(t11, w[6]);
    const float2 t21 = sub2(t14, w[2]);
    const float2 t22 = __fadd2_rn(t16, w[7]);
    const float2 t23 = sub2(t13, w[9]);
    const float2 t24 = __fadd2_rn(t13, w[9]);
    const float2 t25 = sub2(t16, w[7]);
    const float2 t26 = __fadd2_rn(t18, t17);
    const float2 t27 = sub2(t21, t22);
    const float2 t28 = __fadd2_rn(t11, t17);
    const float2 t29 = sub2(t11, t25);
    const float2 t30 = __fadd2_rn(t20, t23);
    const float2 t31 = sub2(t19, t13);
    const float2 t32 = __fadd2_rn(t15, t24);
    const float2 t33 = sub2(t15, t13);
    const float2 t34 = __fadd2_rn(t15, t13);
    const float2 t35 = sub2(t15, t24);
    const float2 t36 = __fadd2_rn(t19, t13);
    const float2 t37 = sub2(t20, t23);
    const float2 t38 = __fadd2_rn(t11, t25);
    const float2 t39 = sub2(t11, t17);
    const float2 t40 = __fadd2_rn(t21, t22);
    const float2 t41 = sub2(t18, t17);
    z[0] = t26;
    z[1] = t28;
    z[2] = t30;
    z[3] = t32;
    z[4] = t34;
    z[5] = t36;
    z[6] = t38;
    z[7] = t40;
    z[8] = t27;
    z[9] = t29;
    z[10] = t31;
    z[11] = t33;
    z[12] = t35;
    z[13] = t37;
    z[14] = t39;
    z[15] = t41;
  }
};

// inverse row pass, inputs v < 16: z[j] = sign[j] * (T^t w)[j]; 44 pair additions
struct InvRow16 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&z)[16]) {
    const float2 t16 = __fadd2_rn(w[0], w[8]);
    const float2 t17 = sub2(w[0], w[8]);
    const float2 t18 = __fadd2_rn(w[1], w[5]);
    const float2 t19 = sub2(w[1], w[5]);
    const float2 t20 = __fadd2_rn(t16, w[4]);
    const float2 t21 = sub2(t17, w[12]);
    const float2 t22 = __fadd2_rn(t17, w[12]);
    const float2 t23 = sub2(t16, w[4]);
    const float2 t24 = sub2(t18, w[3]);
    const float2 t25 = sub2(t19, w[11]);
    const float2 t26 = __fadd2_rn(t19, w[11]);
    const float2 t27 = __fadd2_rn(t18, w[3]);
    const float2 t28 = __fadd2_rn(t20, w[2]);
    const float2 t29 = __fadd2_rn(t23, w[14]);
    const float2 t30 = sub2(t21, w[10]);
    const float2 t31 = __fadd2_rn(t22, w[6]);
    const float2 t32 = sub2(t22, w[6]);
    const float2 t33 = __fadd2_rn(t21, w[10]);
    const float2 t34 = sub2(t23, w[14]);
    const float2 t35 = sub2(t20, w[2]);
    const float2 t36 = __fadd2_rn(t24, w[7]);
    const float2 t37 = sub2(t27, w[13]);
    const float2 t38 = sub2(t25, w[15]);
    const float2 t39 = sub2(t26, w[9]);
    const float2 t40 = __fadd2_rn(t26, w[9]);
    const float2 t41 = __fadd2_rn(t25, w[15]);
    const float2 t42 = __fadd2_rn(t27, w[13]);
    const float2 t43 = sub2(t24, w[7]);
    const float2 t44 = __fadd2_rn(t28, t42);
    const float2 t45 = sub2(t35, t36);
    const float2 t46 = __fadd2_rn(t30, t37);
    const float2 t47 = sub2(t33, t43);
    const float2 t48 = __fadd2_rn(t32, t39);
    const float2 t49 = sub2(t31, t41);
    const float2 t50 = __fadd2_rn(t34, t40);
    const float2 t51 = sub2(t29, t38);
    const float2 t52 = __fadd2_rn(t29, t38);
    const float2 t53 = sub2(t34, t40);
    const float2 t54 = __fadd2_rn(t31, t41);
    const float2 t55 = sub2(t32, t39);
    const float2 t56 = __fadd2_rn(t33, t43);
    const float2 t57 = sub2(t30, t37);
    const float2 t58 = __fadd2_rn(t35, t36);
    const float2 t59 = sub2(t28, t42);
    z[0] = t44;
    z[1] = t46;
    z[2] = t48;
    z[3] = t50;
    z[4] = t52;
    z[5] = t54;
    z[6] = t56;
    z[7] = t58;
    z[8] = t45;
    z[9] = t47;
    z[10] = t49;
    z[11] = t51;
    z[12] = t53;
    z[13] = t55;
    z[14] = t57;
    z[15] = t59;
  }
};

// forward row pass on two rows (lanes: row i, row 15 - i), outputs v < 4, then the
// first column butterfly across the lanes: S[c] = (a_i[2c], a_i[2c+1]) with
// a_i = row i + row 15 - i, D[c] the same for a_(15-i) = row i - row 15 - i (true
// signs); 32 pair additions and 8 scalar additions
struct FwdRowT4 {
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&S)[2], float2 (&D)[2]) {
    const float2 t16 = __fadd2_rn(X[0], X[15]);
    const float2 t17 = sub2(X[7], X[8]);
    const float2 t18 = __fadd2_rn(X[1], X[14]);
    const float2 t19 = sub2(X[6], X[9]);
    const float2 t20 = __fadd2_rn(X[2], X[13]);
    const float2 t21 = sub2(X[5], X[10]);
    const float2 t22 = __fadd2_rn(X[3], X[12]);
    const float2 t23 = sub2(X[4], X[11]);
    const float2 t24 = __fadd2_rn(X[4], X[11]);
    const float2 t25 = sub2(X[3], X[12]);
    const float2 t26 = __fadd2_rn(X[5], X[10]);
    const float2 t27 = sub2(X[2], X[13]);
    const float2 t28 = __fadd2_rn(X[6], X[9]);
    const float2 t29 = sub2(X[1], X[14]);
    const float2 t30 = __fadd2_rn(X[7], X[8]);
    const float2 t31 = sub2(X[0], X[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    S[0] = make_float2(__fadd_rn(t56.x, t56.y), __fadd_rn(t58.x, t58.y));
    D[0] = make_float2(__fadd_rn(t56.x, -t56.y), __fadd_rn(t58.x, -t58.y));
    S[1] = make_float2(__fadd_rn(t39.x, t39.y), __fadd_rn(-t55.x, -t55.y));
    D[1] = make_float2(__fadd_rn(t39.x, -t39.y), __fadd_rn(-t55.x, t55.y));
  }
};

// forward row pass on two rows (lanes: row i, row 15 - i), outputs v < 6, then the
// first column butterfly across the lanes: S[c] = (a_i[2c], a_i[2c+1]) with
// a_i = row i + row 15 - i, D[c] the same for a_(15-i) = row i - row 15 - i (true
// signs); 34 pair additions and 12 scalar additions
struct FwdRowT6 {
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&S)[3], float2 (&D)[3]) {
    const float2 t16 = __fadd2_rn(X[0], X[15]);
    const float2 t17 = sub2(X[7], X[8]);
    const float2 t18 = __fadd2_rn(X[1], X[14]);
    const float2 t19 = sub2(X[6], X[9]);
    const float2 t20 = __fadd2_rn(X[2], X[13]);
    const float2 t21 = sub2(X[5], X[10]);
    const float2 t22 = __fadd2_rn(X[3], X[12]);
    const float2 t23 = sub2(X[4], X[11]);
    const float2 t24 = __fadd2_rn(X[4], X[11]);
    const float2 t25 = sub2(X[3], X[12]);
    const float2 t26 = __fadd2_rn(X[5], X[10]);
    const float2 t27 = sub2(X[2], X[13]);
    const float2 t28 = __fadd2_rn(X[6], X[9]);
    const float2 t29 = sub2(X[1], X[14]);
    const float2 t30 = __fadd2_rn(X[7], X[8]);
    const float2 t31 = sub2(X[0], X[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    S[0] = make_float2(__fadd_rn(t56.x, t56.y), __fadd_rn(t58.x, t58.y));
    D[0] = make_float2(__fadd_rn(t56.x, -t56.y), __fadd_rn(t58.x, -t58.y));
    S[1] = make_float2(__fadd_rn(t39.x, t39.y), __fadd_rn(-t55.x, -t55.y));
    D[1] = make_float2(__fadd_rn(t39.x, -t39.y), __fadd_rn(-t55.x, t55.y));
    S[2] = make_float2(__fadd_rn(t51.x, t51.y), __fadd_rn(t59.x, t59.y));
    D[2] = make_float2(__fadd_rn(t51.x, -t51.y), __fadd_rn(t59.x, -t59.y));
  }
};

// forward row pass on two rows (lanes: row i, row 15 - i), outputs v < 8, then the
// first column butterfly across the lanes: S[c] = (a_i[2c], a_i[2c+1]) with
// a_i = row i + row 15 - i, D[c] the same for a_(15-i) = row i - row 15 - i (true
// signs); 36 pair additions and 16 scalar additions
struct FwdRowT8 {
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&S)[4], float2 (&D)[4]) {
    const float2 t16 = __fadd2_rn(X[0], X[15]);
    const float2 t17 = sub2(X[7], X[8]);
    const float2 t18 = __fadd2_rn(X[1], X[14]);
    const float2 t19 = sub2(X[6], X[9]);
    const float2 t20 = __fadd2_rn(X[2], X[13]);
    const float2 t21 = sub2(X[5], X[10]);
    const float2 t22 = __fadd2_rn(X[3], X[12]);
    const float2 t23 = sub2(X[4], X[11]);
    const float2 t24 = __fadd2_rn(X[4], X[11]);
    const float2 t25 = sub2(X[3], X[12]);
    const float2 t26 = __fadd2_rn(X[5], X[10]);
    const float2 t27 = sub2(X[2], X[13]);
    const float2 t28 = __fadd2_rn(X[6], X[9]);
    const float2 t29 = sub2(X[1], X[14]);
    const float2 t30 = __fadd2_rn(X[7], X[8]);
    const float2 t31 = sub2(X[0], X[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = sub2(t20, t26);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = sub2(t17, t19);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    S[0] = make_float2(__fadd_rn(t56.x, t56.y), __fadd_rn(t58.x, t58.y));
    D[0] = make_float2(__fadd_rn(t56.x, -t56.y), __fadd_rn(t58.x, -t58.y));
    S[1] = make_float2(__fadd_rn(t39.x, t39.y), __fadd_rn(-t55.x, -t55.y));
    D[1] = make_float2(__fadd_rn(t39.x, -t39.y), __fadd_rn(-t55.x, t55.y));
    S[2] = make_float2(__fadd_rn(t51.x, t51.y), __fadd_rn(t59.x, t59.y));
    D[2] = make_float2(__fadd_rn(t51.x, -t51.y), __fadd_rn(t59.x, -t59.y));
    S[3] = make_float2(__fadd_rn(-t35.x, -t35.y), __fadd_rn(t47.x, t47.y));
    D[3] = make_float2(__fadd_rn(-t35.x, t35.y), __fadd_rn(t47.x, -t47.y));
  }
};

// forward row pass on two rows (lanes: row i, row 15 - i), outputs v < 10, then the
// first column butterfly across the lanes: S[c] = (a_i[2c], a_i[2c+1]) with
// a_i = row i + row 15 - i, D[c] the same for a_(15-i) = row i - row 15 - i (true
// signs); 38 pair additions and 20 scalar additions
struct FwdRowT10 {
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&S)[5], float2 (&D)[5]) {
    const float2 t16 = __fadd2_rn(X[0], X[15]);
    const float2 t17 = sub2(X[7], X[8]);
    const float2 t18 = __fadd2_rn(X[1], X[14]);
    const float2 t19 = sub2(X[6], X[9]);
    const float2 t20 = __fadd2_rn(X[2], X[13]);
    const float2 t21 = sub2(X[5], X[10]);
    const float2 t22 = __fadd2_rn(X[3], X[12]);
    const float2 t23 = sub2(X[4], X[11]);
    const float2 t24 = __fadd2_rn(X[4], X[11]);
    const float2 t25 = sub2(X[3], X[12]);
    const float2 t26 = __fadd2_rn(X[5], X[10]);
    const float2 t27 = sub2(X[2], X[13]);
    const float2 t28 = __fadd2_rn(X[6], X[9]);
    const float2 t29 = sub2(X[1], X[14]);
    const float2 t30 = __fadd2_rn(X[7], X[8]);
    const float2 t31 = sub2(X[0], X[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = sub2(t20, t26);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t43 = sub2(t25, t27);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = sub2(t17, t19);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t57 = sub2(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    S[0] = make_float2(__fadd_rn(t56.x, t56.y), __fadd_rn(t58.x, t58.y));
    D[0] = make_float2(__fadd_rn(t56.x, -t56.y), __fadd_rn(t58.x, -t58.y));
    S[1] = make_float2(__fadd_rn(t39.x, t39.y), __fadd_rn(-t55.x, -t55.y));
    D[1] = make_float2(__fadd_rn(t39.x, -t39.y), __fadd_rn(-t55.x, t55.y));
    S[2] = make_float2(__fadd_rn(t51.x, t51.y), __fadd_rn(t59.x, t59.y));
    D[2] = make_float2(__fadd_rn(t51.x, -t51.y), __fadd_rn(t59.x, -t59.y));
    S[3] = make_float2(__fadd_rn(-t35.x, -t35.y), __fadd_rn(t47.x, t47.y));
    D[3] = make_float2(__fadd_rn(-t35.x, t35.y), __fadd_rn(t47.x, -t47.y));
    S[4] = make_float2(__fadd_rn(t57.x, t57.y), __fadd_rn(t43.x, t43.y));
    D[4] = make_float2(__fadd_rn(t57.x, -t57.y), __fadd_rn(t43.x, -t43.y));
  }
};

// forward row pass on two rows (lanes: row i, row 15 - i), outputs v < 16, then the
// first column butterfly across the lanes: S[c] = (a_i[2c], a_i[2c+1]) with
// a_i = row i + row 15 - i, D[c] the same for a_(15-i) = row i - row 15 - i (true
// signs); 44 pair additions and 32 scalar additions
struct FwdRowT16 {
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&S)[8], float2 (&D)[8]) {
    const float2 t16 = __fadd2_rn(X[0], X[15]);
    const float2 t17 = sub2(X[7], X[8]);
    const float2 t18 = __fadd2_rn(X[1], X[14]);
    const float2 t19 = sub2(X[6], X[9]);
    const float2 t20 = __fadd2_rn(X[2], X[13]);
    const float2 t21 = sub2(X[5], X[10]);
    const float2 t22 = __fadd2_rn(X[3], X[12]);
    const float2 t23 = sub2(X[4], X[11]);
    const float2 t24 = __fadd2_rn(X[4], X[11]);
    const float2 t25 = sub2(X[3], X[12]);
    const float2 t26 = __fadd2_rn(X[5], X[10]);
    const float2 t27 = sub2(X[2], X[13]);
    const float2 t28 = __fadd2_rn(X[6], X[9]);
    const float2 t29 = sub2(X[1], X[14]);
    const float2 t30 = __fadd2_rn(X[7], X[8]);
    const float2 t31 = sub2(X[0], X[15]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t33 = sub2(t22, t24);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = sub2(t20, t26);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t37 = sub2(t18, t28);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = sub2(t16, t30);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t41 = sub2(t29, t31);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t43 = sub2(t25, t27);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t45 = sub2(t21, t23);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = sub2(t17, t19);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t50 = sub2(t34, t36);
    const float2 t51 = sub2(t32, t38);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t54 = sub2(t42, t44);
    const float2 t55 = sub2(t40, t46);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t57 = sub2(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = sub2(t52, t53);
    S[0] = make_float2(__fadd_rn(t56.x, t56.y), __fadd_rn(t58.x, t58.y));
    D[0] = make_float2(__fadd_rn(t56.x, -t56.y), __fadd_rn(t58.x, -t58.y));
    S[1] = make_float2(__fadd_rn(t39.x, t39.y), __fadd_rn(-t55.x, -t55.y));
    D[1] = make_float2(__fadd_rn(t39.x, -t39.y), __fadd_rn(-t55.x, t55.y));
    S[2] = make_float2(__fadd_rn(t51.x, t51.y), __fadd_rn(t59.x, t59.y));
    D[2] = make_float2(__fadd_rn(t51.x, -t51.y), __fadd_rn(t59.x, -t59.y));
    S[3] = make_float2(__fadd_rn(-t35.x, -t35.y), __fadd_rn(t47.x, t47.y));
    D[3] = make_float2(__fadd_rn(-t35.x, t35.y), __fadd_rn(t47.x, -t47.y));
    S[4] = make_float2(__fadd_rn(t57.x, t57.y), __fadd_rn(t43.x, t43.y));
    D[4] = make_float2(__fadd_rn(t57.x, -t57.y), __fadd_rn(t43.x, -t43.y));
    S[5] = make_float2(__fadd_rn(-t37.x, -t37.y), __fadd_rn(-t54.x, -t54.y));
    D[5] = make_float2(__fadd_rn(-t37.x, t37.y), __fadd_rn(-t54.x, t54.y));
    S[6] = make_float2(__fadd_rn(-t50.x, -t50.y), __fadd_rn(-t41.x, -t41.y));
    D[6] = make_float2(__fadd_rn(-t50.x, t50.y), __fadd_rn(-t41.x, t41.y));
    S[7] = make_float2(__fadd_rn(-t33.x, -t33.y), __fadd_rn(t45.x, t45.y));
    D[7] = make_float2(__fadd_rn(-t33.x, t33.y), __fadd_rn(t45.x, -t45.y));
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 1:
// n[u] = sign[u] * (T x)[u]; 7 pair additions
struct FwdColM1 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfffeu, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[1]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t40 = __fadd2_rn(t32, t33);
    n[0] = t40;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 2:
// n[u] = sign[u] * (T x)[u]; 14 pair additions
struct FwdColM2 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfffcu, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[2]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    n[0] = t40;
    n[1] = t42;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 3:
// n[u] = sign[u] * (T x)[u]; 15 pair additions
struct FwdColM3 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfff8u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[3]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 4:
// n[u] = sign[u] * (T x)[u]; 16 pair additions
struct FwdColM4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xfff0u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[4]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 5:
// n[u] = sign[u] * (T x)[u]; 17 pair additions
struct FwdColM5 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xffe0u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[5]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 6:
// n[u] = sign[u] * (T x)[u]; 18 pair additions
struct FwdColM6 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xffc0u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[6]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 7:
// n[u] = sign[u] * (T x)[u]; 19 pair additions
struct FwdColM7 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xff80u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[7]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 8:
// n[u] = sign[u] * (T x)[u]; 20 pair additions
struct FwdColM8 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[8]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 9:
// n[u] = sign[u] * (T x)[u]; 21 pair additions
struct FwdColM9 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xfe00u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[9]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 10:
// n[u] = sign[u] * (T x)[u]; 22 pair additions
struct FwdColM10 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0048u, 0xfc00u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[10]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 11:
// n[u] = sign[u] * (T x)[u]; 23 pair additions
struct FwdColM11 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0448u, 0xf800u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[11]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t21 = sub2(a[1], a[6]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
    n[10] = t21;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 12:
// n[u] = sign[u] * (T x)[u]; 24 pair additions
struct FwdColM12 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0c48u, 0xf000u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[12]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t21 = sub2(a[1], a[6]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = sub2(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
    n[10] = t21;
    n[11] = t38;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 13:
// n[u] = sign[u] * (T x)[u]; 25 pair additions
struct FwdColM13 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x1c48u, 0xe000u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[13]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t21 = sub2(a[1], a[6]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t34 = sub2(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = sub2(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
    n[10] = t21;
    n[11] = t38;
    n[12] = t34;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 14:
// n[u] = sign[u] * (T x)[u]; 26 pair additions
struct FwdColM14 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x3c48u, 0xc000u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[14]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t21 = sub2(a[1], a[6]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t25 = sub2(a[14], a[15]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t34 = sub2(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = sub2(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
    n[10] = t21;
    n[11] = t38;
    n[12] = t34;
    n[13] = t25;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 15:
// n[u] = sign[u] * (T x)[u]; 27 pair additions
struct FwdColM15 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x7c48u, 0x8000u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[15]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t17 = sub2(a[3], a[4]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t21 = sub2(a[1], a[6]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t25 = sub2(a[14], a[15]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t34 = sub2(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = sub2(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
    n[10] = t21;
    n[11] = t38;
    n[12] = t34;
    n[13] = t25;
    n[14] = t17;
  }
};

// forward column pass after M1 (inputs a = M1 x), outputs u < 16:
// n[u] = sign[u] * (T x)[u]; 28 pair additions
struct FwdColM16 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x7c48u, 0x0000u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[16], float2 (&n)[16]) {
    const float2 t16 = __fadd2_rn(a[0], a[7]);
    const float2 t17 = sub2(a[3], a[4]);
    const float2 t18 = __fadd2_rn(a[1], a[6]);
    const float2 t19 = sub2(a[2], a[5]);
    const float2 t20 = __fadd2_rn(a[2], a[5]);
    const float2 t21 = sub2(a[1], a[6]);
    const float2 t22 = __fadd2_rn(a[3], a[4]);
    const float2 t23 = sub2(a[0], a[7]);
    const float2 t24 = __fadd2_rn(a[8], a[9]);
    const float2 t25 = sub2(a[14], a[15]);
    const float2 t26 = __fadd2_rn(a[11], a[10]);
    const float2 t27 = sub2(a[12], a[13]);
    const float2 t28 = __fadd2_rn(a[12], a[13]);
    const float2 t29 = sub2(a[10], a[11]);
    const float2 t30 = __fadd2_rn(a[15], a[14]);
    const float2 t31 = sub2(a[8], a[9]);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t34 = sub2(t18, t20);
    const float2 t35 = sub2(t16, t22);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = sub2(t26, t28);
    const float2 t39 = sub2(t24, t30);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = sub2(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = sub2(t36, t37);
    n[0] = t40;
    n[1] = t42;
    n[2] = t23;
    n[3] = t39;
    n[4] = t35;
    n[5] = t43;
    n[6] = t19;
    n[7] = t31;
    n[8] = t41;
    n[9] = t27;
    n[10] = t21;
    n[11] = t38;
    n[12] = t34;
    n[13] = t25;
    n[14] = t17;
    n[15] = t29;
  }
};

// inverse column pass, inputs u < 1 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 0 pair additions and 0 scalar additions
struct InvColT1 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    Z[0][0] = make_float2(w[0].x, w[0].x);
    Z[0][1] = make_float2(w[0].y, w[0].y);
    Z[1][0] = make_float2(w[0].x, w[0].x);
    Z[1][1] = make_float2(w[0].y, w[0].y);
    Z[2][0] = make_float2(w[0].x, w[0].x);
    Z[2][1] = make_float2(w[0].y, w[0].y);
    Z[3][0] = make_float2(w[0].x, w[0].x);
    Z[3][1] = make_float2(w[0].y, w[0].y);
    Z[4][0] = make_float2(w[0].x, w[0].x);
    Z[4][1] = make_float2(w[0].y, w[0].y);
    Z[5][0] = make_float2(w[0].x, w[0].x);
    Z[5][1] = make_float2(w[0].y, w[0].y);
    Z[6][0] = make_float2(w[0].x, w[0].x);
    Z[6][1] = make_float2(w[0].y, w[0].y);
    Z[7][0] = make_float2(w[0].x, w[0].x);
    Z[7][1] = make_float2(w[0].y, w[0].y);
  }
};

// inverse column pass, inputs u < 2 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 0 pair additions and 4 scalar additions
struct InvColT2 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float s0 = __fadd_rn(w[0].x, w[1].x);
    const float s1 = __fadd_rn(-w[1].x, w[0].x);
    const float s2 = __fadd_rn(w[0].y, w[1].y);
    const float s3 = __fadd_rn(-w[1].y, w[0].y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s0, s1);
    Z[1][1] = make_float2(s2, s3);
    Z[2][0] = make_float2(s0, s1);
    Z[2][1] = make_float2(s2, s3);
    Z[3][0] = make_float2(s0, s1);
    Z[3][1] = make_float2(s2, s3);
    Z[4][0] = make_float2(s0, s1);
    Z[4][1] = make_float2(s2, s3);
    Z[5][0] = make_float2(s0, s1);
    Z[5][1] = make_float2(s2, s3);
    Z[6][0] = make_float2(s0, s1);
    Z[6][1] = make_float2(s2, s3);
    Z[7][0] = make_float2(s0, s1);
    Z[7][1] = make_float2(s2, s3);
  }
};

// inverse column pass, inputs u < 3 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 2 pair additions and 12 scalar additions
struct InvColT3 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t3 = __fadd2_rn(w[0], w[2]);
    const float2 t4 = sub2(w[0], w[2]);
    const float s0 = __fadd_rn(t3.x, w[1].x);
    const float s1 = __fadd_rn(-w[1].x, t3.x);
    const float s2 = __fadd_rn(t3.y, w[1].y);
    const float s3 = __fadd_rn(-w[1].y, t3.y);
    const float s4 = __fadd_rn(w[0].x, w[1].x);
    const float s5 = __fadd_rn(-w[1].x, w[0].x);
    const float s6 = __fadd_rn(w[0].y, w[1].y);
    const float s7 = __fadd_rn(-w[1].y, w[0].y);
    const float s8 = __fadd_rn(t4.x, w[1].x);
    const float s9 = __fadd_rn(-w[1].x, t4.x);
    const float s10 = __fadd_rn(t4.y, w[1].y);
    const float s11 = __fadd_rn(-w[1].y, t4.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s4, s5);
    Z[2][1] = make_float2(s6, s7);
    Z[3][0] = make_float2(s4, s5);
    Z[3][1] = make_float2(s6, s7);
    Z[4][0] = make_float2(s4, s5);
    Z[4][1] = make_float2(s6, s7);
    Z[5][0] = make_float2(s4, s5);
    Z[5][1] = make_float2(s6, s7);
    Z[6][0] = make_float2(s4, s5);
    Z[6][1] = make_float2(s6, s7);
    Z[7][0] = make_float2(s8, s9);
    Z[7][1] = make_float2(s10, s11);
  }
};

// inverse column pass, inputs u < 4 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 4 pair additions and 20 scalar additions
struct InvColT4 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t4 = sub2(w[1], w[3]);
    const float2 t5 = __fadd2_rn(w[1], w[3]);
    const float2 t6 = __fadd2_rn(w[0], w[2]);
    const float2 t7 = sub2(w[0], w[2]);
    const float s0 = __fadd_rn(t5.x, t6.x);
    const float s1 = __fadd_rn(-t5.x, t6.x);
    const float s2 = __fadd_rn(t5.y, t6.y);
    const float s3 = __fadd_rn(-t5.y, t6.y);
    const float s4 = __fadd_rn(t5.x, w[0].x);
    const float s5 = __fadd_rn(-t5.x, w[0].x);
    const float s6 = __fadd_rn(t5.y, w[0].y);
    const float s7 = __fadd_rn(-t5.y, w[0].y);
    const float s8 = __fadd_rn(w[0].x, w[1].x);
    const float s9 = __fadd_rn(-w[1].x, w[0].x);
    const float s10 = __fadd_rn(w[0].y, w[1].y);
    const float s11 = __fadd_rn(-w[1].y, w[0].y);
    const float s12 = __fadd_rn(t4.x, w[0].x);
    const float s13 = __fadd_rn(-t4.x, w[0].x);
    const float s14 = __fadd_rn(t4.y, w[0].y);
    const float s15 = __fadd_rn(-t4.y, w[0].y);
    const float s16 = __fadd_rn(t4.x, t7.x);
    const float s17 = __fadd_rn(-t4.x, t7.x);
    const float s18 = __fadd_rn(t4.y, t7.y);
    const float s19 = __fadd_rn(-t4.y, t7.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s8, s9);
    Z[3][1] = make_float2(s10, s11);
    Z[4][0] = make_float2(s8, s9);
    Z[4][1] = make_float2(s10, s11);
    Z[5][0] = make_float2(s8, s9);
    Z[5][1] = make_float2(s10, s11);
    Z[6][0] = make_float2(s12, s13);
    Z[6][1] = make_float2(s14, s15);
    Z[7][0] = make_float2(s16, s17);
    Z[7][1] = make_float2(s18, s19);
  }
};

// inverse column pass, inputs u < 5 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 6 pair additions and 24 scalar additions
struct InvColT5 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t5 = __fadd2_rn(w[0], w[4]);
    const float2 t6 = sub2(w[0], w[4]);
    const float2 t7 = sub2(w[1], w[3]);
    const float2 t8 = __fadd2_rn(w[1], w[3]);
    const float2 t9 = __fadd2_rn(t5, w[2]);
    const float2 t10 = sub2(w[2], t5);
    const float s0 = __fadd_rn(t8.x, t9.x);
    const float s1 = __fadd_rn(-t8.x, t9.x);
    const float s2 = __fadd_rn(t8.y, t9.y);
    const float s3 = __fadd_rn(-t8.y, t9.y);
    const float s4 = __fadd_rn(t8.x, w[0].x);
    const float s5 = __fadd_rn(-t8.x, w[0].x);
    const float s6 = __fadd_rn(t8.y, w[0].y);
    const float s7 = __fadd_rn(-t8.y, w[0].y);
    const float s8 = __fadd_rn(w[0].x, w[1].x);
    const float s9 = __fadd_rn(-w[1].x, w[0].x);
    const float s10 = __fadd_rn(w[0].y, w[1].y);
    const float s11 = __fadd_rn(-w[1].y, w[0].y);
    const float s12 = __fadd_rn(t6.x, w[1].x);
    const float s13 = __fadd_rn(-w[1].x, t6.x);
    const float s14 = __fadd_rn(t6.y, w[1].y);
    const float s15 = __fadd_rn(-w[1].y, t6.y);
    const float s16 = __fadd_rn(t7.x, w[0].x);
    const float s17 = __fadd_rn(-t7.x, w[0].x);
    const float s18 = __fadd_rn(t7.y, w[0].y);
    const float s19 = __fadd_rn(-t7.y, w[0].y);
    const float s20 = __fadd_rn(-t10.x, t7.x);
    const float s21 = __fadd_rn(-t10.x, -t7.x);
    const float s22 = __fadd_rn(-t10.y, t7.y);
    const float s23 = __fadd_rn(-t10.y, -t7.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s12, s13);
    Z[4][1] = make_float2(s14, s15);
    Z[5][0] = make_float2(s8, s9);
    Z[5][1] = make_float2(s10, s11);
    Z[6][0] = make_float2(s16, s17);
    Z[6][1] = make_float2(s18, s19);
    Z[7][0] = make_float2(s20, s21);
    Z[7][1] = make_float2(s22, s23);
  }
};

// inverse column pass, inputs u < 6 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 8 pair additions and 24 scalar additions
struct InvColT6 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t6 = __fadd2_rn(w[1], w[5]);
    const float2 t7 = sub2(w[1], w[5]);
    const float2 t8 = __fadd2_rn(w[0], w[4]);
    const float2 t9 = sub2(w[0], w[4]);
    const float2 t10 = sub2(w[3], t6);
    const float2 t11 = __fadd2_rn(t6, w[3]);
    const float2 t12 = __fadd2_rn(t8, w[2]);
    const float2 t13 = sub2(w[2], t8);
    const float s0 = __fadd_rn(t11.x, t12.x);
    const float s1 = __fadd_rn(-t11.x, t12.x);
    const float s2 = __fadd_rn(t11.y, t12.y);
    const float s3 = __fadd_rn(-t11.y, t12.y);
    const float s4 = __fadd_rn(t11.x, w[0].x);
    const float s5 = __fadd_rn(-t11.x, w[0].x);
    const float s6 = __fadd_rn(t11.y, w[0].y);
    const float s7 = __fadd_rn(-t11.y, w[0].y);
    const float s8 = __fadd_rn(t7.x, w[0].x);
    const float s9 = __fadd_rn(-t7.x, w[0].x);
    const float s10 = __fadd_rn(t7.y, w[0].y);
    const float s11 = __fadd_rn(-t7.y, w[0].y);
    const float s12 = __fadd_rn(t7.x, t9.x);
    const float s13 = __fadd_rn(-t7.x, t9.x);
    const float s14 = __fadd_rn(t7.y, t9.y);
    const float s15 = __fadd_rn(-t7.y, t9.y);
    const float s16 = __fadd_rn(-t10.x, w[0].x);
    const float s17 = __fadd_rn(t10.x, w[0].x);
    const float s18 = __fadd_rn(-t10.y, w[0].y);
    const float s19 = __fadd_rn(t10.y, w[0].y);
    const float s20 = __fadd_rn(-t10.x, -t13.x);
    const float s21 = __fadd_rn(-t13.x, t10.x);
    const float s22 = __fadd_rn(-t10.y, -t13.y);
    const float s23 = __fadd_rn(-t13.y, t10.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s12, s13);
    Z[4][1] = make_float2(s14, s15);
    Z[5][0] = make_float2(s8, s9);
    Z[5][1] = make_float2(s10, s11);
    Z[6][0] = make_float2(s16, s17);
    Z[6][1] = make_float2(s18, s19);
    Z[7][0] = make_float2(s20, s21);
    Z[7][1] = make_float2(s22, s23);
  }
};

// inverse column pass, inputs u < 7 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 10 pair additions and 28 scalar additions
struct InvColT7 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t7 = __fadd2_rn(w[1], w[5]);
    const float2 t8 = sub2(w[1], w[5]);
    const float2 t9 = __fadd2_rn(w[0], w[4]);
    const float2 t10 = sub2(w[0], w[4]);
    const float2 t11 = sub2(w[3], t7);
    const float2 t12 = __fadd2_rn(t7, w[3]);
    const float2 t13 = __fadd2_rn(t9, w[2]);
    const float2 t14 = __fadd2_rn(w[0], w[6]);
    const float2 t15 = sub2(w[0], w[6]);
    const float2 t16 = sub2(w[2], t9);
    const float s0 = __fadd_rn(t12.x, t13.x);
    const float s1 = __fadd_rn(-t12.x, t13.x);
    const float s2 = __fadd_rn(t12.y, t13.y);
    const float s3 = __fadd_rn(-t12.y, t13.y);
    const float s4 = __fadd_rn(t12.x, w[0].x);
    const float s5 = __fadd_rn(-t12.x, w[0].x);
    const float s6 = __fadd_rn(t12.y, w[0].y);
    const float s7 = __fadd_rn(-t12.y, w[0].y);
    const float s8 = __fadd_rn(t15.x, t8.x);
    const float s9 = __fadd_rn(-t8.x, t15.x);
    const float s10 = __fadd_rn(t15.y, t8.y);
    const float s11 = __fadd_rn(-t8.y, t15.y);
    const float s12 = __fadd_rn(t10.x, t8.x);
    const float s13 = __fadd_rn(-t8.x, t10.x);
    const float s14 = __fadd_rn(t10.y, t8.y);
    const float s15 = __fadd_rn(-t8.y, t10.y);
    const float s16 = __fadd_rn(t14.x, t8.x);
    const float s17 = __fadd_rn(-t8.x, t14.x);
    const float s18 = __fadd_rn(t14.y, t8.y);
    const float s19 = __fadd_rn(-t8.y, t14.y);
    const float s20 = __fadd_rn(-t11.x, w[0].x);
    const float s21 = __fadd_rn(t11.x, w[0].x);
    const float s22 = __fadd_rn(-t11.y, w[0].y);
    const float s23 = __fadd_rn(t11.y, w[0].y);
    const float s24 = __fadd_rn(-t11.x, -t16.x);
    const float s25 = __fadd_rn(-t16.x, t11.x);
    const float s26 = __fadd_rn(-t11.y, -t16.y);
    const float s27 = __fadd_rn(-t16.y, t11.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s12, s13);
    Z[4][1] = make_float2(s14, s15);
    Z[5][0] = make_float2(s16, s17);
    Z[5][1] = make_float2(s18, s19);
    Z[6][0] = make_float2(s20, s21);
    Z[6][1] = make_float2(s22, s23);
    Z[7][0] = make_float2(s24, s25);
    Z[7][1] = make_float2(s26, s27);
  }
};

// inverse column pass, inputs u < 8 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 12 pair additions and 28 scalar additions
struct InvColT8 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t8 = __fadd2_rn(w[1], w[5]);
    const float2 t9 = sub2(w[1], w[5]);
    const float2 t10 = __fadd2_rn(w[0], w[4]);
    const float2 t11 = sub2(w[0], w[4]);
    const float2 t12 = sub2(w[3], t8);
    const float2 t13 = __fadd2_rn(t8, w[3]);
    const float2 t14 = __fadd2_rn(t10, w[2]);
    const float2 t15 = __fadd2_rn(w[0], w[6]);
    const float2 t16 = sub2(w[0], w[6]);
    const float2 t17 = sub2(w[2], t10);
    const float2 t18 = sub2(w[7], t12);
    const float2 t19 = __fadd2_rn(t12, w[7]);
    const float s0 = __fadd_rn(t13.x, t14.x);
    const float s1 = __fadd_rn(-t13.x, t14.x);
    const float s2 = __fadd_rn(t13.y, t14.y);
    const float s3 = __fadd_rn(-t13.y, t14.y);
    const float s4 = __fadd_rn(t13.x, w[0].x);
    const float s5 = __fadd_rn(-t13.x, w[0].x);
    const float s6 = __fadd_rn(t13.y, w[0].y);
    const float s7 = __fadd_rn(-t13.y, w[0].y);
    const float s8 = __fadd_rn(t16.x, t9.x);
    const float s9 = __fadd_rn(-t9.x, t16.x);
    const float s10 = __fadd_rn(t16.y, t9.y);
    const float s11 = __fadd_rn(-t9.y, t16.y);
    const float s12 = __fadd_rn(t11.x, t9.x);
    const float s13 = __fadd_rn(-t9.x, t11.x);
    const float s14 = __fadd_rn(t11.y, t9.y);
    const float s15 = __fadd_rn(-t9.y, t11.y);
    const float s16 = __fadd_rn(t15.x, t9.x);
    const float s17 = __fadd_rn(-t9.x, t15.x);
    const float s18 = __fadd_rn(t15.y, t9.y);
    const float s19 = __fadd_rn(-t9.y, t15.y);
    const float s20 = __fadd_rn(-t19.x, w[0].x);
    const float s21 = __fadd_rn(t19.x, w[0].x);
    const float s22 = __fadd_rn(-t19.y, w[0].y);
    const float s23 = __fadd_rn(t19.y, w[0].y);
    const float s24 = __fadd_rn(-t17.x, t18.x);
    const float s25 = __fadd_rn(-t17.x, -t18.x);
    const float s26 = __fadd_rn(-t17.y, t18.y);
    const float s27 = __fadd_rn(-t17.y, -t18.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s12, s13);
    Z[4][1] = make_float2(s14, s15);
    Z[5][0] = make_float2(s16, s17);
    Z[5][1] = make_float2(s18, s19);
    Z[6][0] = make_float2(s20, s21);
    Z[6][1] = make_float2(s22, s23);
    Z[7][0] = make_float2(s24, s25);
    Z[7][1] = make_float2(s26, s27);
  }
};

// inverse column pass, inputs u < 9 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 14 pair additions and 28 scalar additions
struct InvColT9 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t9 = __fadd2_rn(w[0], w[8]);
    const float2 t10 = sub2(w[0], w[8]);
    const float2 t11 = __fadd2_rn(w[1], w[5]);
    const float2 t12 = sub2(w[1], w[5]);
    const float2 t13 = __fadd2_rn(t9, w[4]);
    const float2 t14 = sub2(w[4], t9);
    const float2 t15 = sub2(w[3], t11);
    const float2 t16 = __fadd2_rn(t11, w[3]);
    const float2 t17 = __fadd2_rn(t13, w[2]);
    const float2 t18 = __fadd2_rn(t10, w[6]);
    const float2 t19 = sub2(w[6], t10);
    const float2 t20 = sub2(w[2], t13);
    const float2 t21 = sub2(w[7], t15);
    const float2 t22 = __fadd2_rn(t15, w[7]);
    const float s0 = __fadd_rn(t16.x, t17.x);
    const float s1 = __fadd_rn(-t16.x, t17.x);
    const float s2 = __fadd_rn(t16.y, t17.y);
    const float s3 = __fadd_rn(-t16.y, t17.y);
    const float s4 = __fadd_rn(t10.x, t16.x);
    const float s5 = __fadd_rn(-t16.x, t10.x);
    const float s6 = __fadd_rn(t10.y, t16.y);
    const float s7 = __fadd_rn(-t16.y, t10.y);
    const float s8 = __fadd_rn(-t19.x, t12.x);
    const float s9 = __fadd_rn(-t12.x, -t19.x);
    const float s10 = __fadd_rn(-t19.y, t12.y);
    const float s11 = __fadd_rn(-t12.y, -t19.y);
    const float s12 = __fadd_rn(-t14.x, t12.x);
    const float s13 = __fadd_rn(-t12.x, -t14.x);
    const float s14 = __fadd_rn(-t14.y, t12.y);
    const float s15 = __fadd_rn(-t12.y, -t14.y);
    const float s16 = __fadd_rn(t12.x, t18.x);
    const float s17 = __fadd_rn(-t12.x, t18.x);
    const float s18 = __fadd_rn(t12.y, t18.y);
    const float s19 = __fadd_rn(-t12.y, t18.y);
    const float s20 = __fadd_rn(-t22.x, t10.x);
    const float s21 = __fadd_rn(t10.x, t22.x);
    const float s22 = __fadd_rn(-t22.y, t10.y);
    const float s23 = __fadd_rn(t10.y, t22.y);
    const float s24 = __fadd_rn(-t20.x, t21.x);
    const float s25 = __fadd_rn(-t20.x, -t21.x);
    const float s26 = __fadd_rn(-t20.y, t21.y);
    const float s27 = __fadd_rn(-t20.y, -t21.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s12, s13);
    Z[4][1] = make_float2(s14, s15);
    Z[5][0] = make_float2(s16, s17);
    Z[5][1] = make_float2(s18, s19);
    Z[6][0] = make_float2(s20, s21);
    Z[6][1] = make_float2(s22, s23);
    Z[7][0] = make_float2(s24, s25);
    Z[7][1] = make_float2(s26, s27);
  }
};

// inverse column pass, inputs u < 10 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 16 pair additions and 32 scalar additions
struct InvColT10 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t10 = __fadd2_rn(w[0], w[8]);
    const float2 t11 = sub2(w[0], w[8]);
    const float2 t12 = __fadd2_rn(w[1], w[5]);
    const float2 t13 = sub2(w[1], w[5]);
    const float2 t14 = __fadd2_rn(t10, w[4]);
    const float2 t15 = sub2(w[4], t10);
    const float2 t16 = sub2(w[3], t12);
    const float2 t17 = __fadd2_rn(t12, w[3]);
    const float2 t18 = __fadd2_rn(t14, w[2]);
    const float2 t19 = __fadd2_rn(t11, w[6]);
    const float2 t20 = sub2(w[6], t11);
    const float2 t21 = sub2(w[2], t14);
    const float2 t22 = sub2(w[7], t16);
    const float2 t23 = sub2(w[9], t13);
    const float2 t24 = __fadd2_rn(t13, w[9]);
    const float2 t25 = __fadd2_rn(t16, w[7]);
    const float s0 = __fadd_rn(t17.x, t18.x);
    const float s1 = __fadd_rn(-t17.x, t18.x);
    const float s2 = __fadd_rn(t17.y, t18.y);
    const float s3 = __fadd_rn(-t17.y, t18.y);
    const float s4 = __fadd_rn(t11.x, t17.x);
    const float s5 = __fadd_rn(-t17.x, t11.x);
    const float s6 = __fadd_rn(t11.y, t17.y);
    const float s7 = __fadd_rn(-t17.y, t11.y);
    const float s8 = __fadd_rn(-t20.x, -t23.x);
    const float s9 = __fadd_rn(-t20.x, t23.x);
    const float s10 = __fadd_rn(-t20.y, -t23.y);
    const float s11 = __fadd_rn(-t20.y, t23.y);
    const float s12 = __fadd_rn(-t15.x, t24.x);
    const float s13 = __fadd_rn(-t15.x, -t24.x);
    const float s14 = __fadd_rn(-t15.y, t24.y);
    const float s15 = __fadd_rn(-t15.y, -t24.y);
    const float s16 = __fadd_rn(-t15.x, t13.x);
    const float s17 = __fadd_rn(-t13.x, -t15.x);
    const float s18 = __fadd_rn(-t15.y, t13.y);
    const float s19 = __fadd_rn(-t13.y, -t15.y);
    const float s20 = __fadd_rn(t13.x, t19.x);
    const float s21 = __fadd_rn(-t13.x, t19.x);
    const float s22 = __fadd_rn(t13.y, t19.y);
    const float s23 = __fadd_rn(-t13.y, t19.y);
    const float s24 = __fadd_rn(-t25.x, t11.x);
    const float s25 = __fadd_rn(t11.x, t25.x);
    const float s26 = __fadd_rn(-t25.y, t11.y);
    const float s27 = __fadd_rn(t11.y, t25.y);
    const float s28 = __fadd_rn(-t21.x, t22.x);
    const float s29 = __fadd_rn(-t21.x, -t22.x);
    const float s30 = __fadd_rn(-t21.y, t22.y);
    const float s31 = __fadd_rn(-t21.y, -t22.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// inverse column pass, inputs u < 11 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 18 pair additions and 32 scalar additions
struct InvColT11 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t11 = __fadd2_rn(w[0], w[8]);
    const float2 t12 = sub2(w[0], w[8]);
    const float2 t13 = __fadd2_rn(w[1], w[5]);
    const float2 t14 = sub2(w[1], w[5]);
    const float2 t15 = __fadd2_rn(t11, w[4]);
    const float2 t16 = sub2(w[4], t11);
    const float2 t17 = sub2(w[3], t13);
    const float2 t18 = __fadd2_rn(t13, w[3]);
    const float2 t19 = __fadd2_rn(t15, w[2]);
    const float2 t20 = sub2(w[10], t12);
    const float2 t21 = __fadd2_rn(t12, w[6]);
    const float2 t22 = sub2(w[6], t12);
    const float2 t23 = __fadd2_rn(t12, w[10]);
    const float2 t24 = sub2(w[2], t15);
    const float2 t25 = sub2(w[7], t17);
    const float2 t26 = sub2(w[9], t14);
    const float2 t27 = __fadd2_rn(t14, w[9]);
    const float2 t28 = __fadd2_rn(t17, w[7]);
    const float s0 = __fadd_rn(t18.x, t19.x);
    const float s1 = __fadd_rn(-t18.x, t19.x);
    const float s2 = __fadd_rn(t18.y, t19.y);
    const float s3 = __fadd_rn(-t18.y, t19.y);
    const float s4 = __fadd_rn(-t20.x, t18.x);
    const float s5 = __fadd_rn(-t18.x, -t20.x);
    const float s6 = __fadd_rn(-t20.y, t18.y);
    const float s7 = __fadd_rn(-t18.y, -t20.y);
    const float s8 = __fadd_rn(-t22.x, -t26.x);
    const float s9 = __fadd_rn(-t22.x, t26.x);
    const float s10 = __fadd_rn(-t22.y, -t26.y);
    const float s11 = __fadd_rn(-t22.y, t26.y);
    const float s12 = __fadd_rn(-t16.x, t27.x);
    const float s13 = __fadd_rn(-t16.x, -t27.x);
    const float s14 = __fadd_rn(-t16.y, t27.y);
    const float s15 = __fadd_rn(-t16.y, -t27.y);
    const float s16 = __fadd_rn(-t16.x, t14.x);
    const float s17 = __fadd_rn(-t14.x, -t16.x);
    const float s18 = __fadd_rn(-t16.y, t14.y);
    const float s19 = __fadd_rn(-t14.y, -t16.y);
    const float s20 = __fadd_rn(t14.x, t21.x);
    const float s21 = __fadd_rn(-t14.x, t21.x);
    const float s22 = __fadd_rn(t14.y, t21.y);
    const float s23 = __fadd_rn(-t14.y, t21.y);
    const float s24 = __fadd_rn(-t28.x, t23.x);
    const float s25 = __fadd_rn(t23.x, t28.x);
    const float s26 = __fadd_rn(-t28.y, t23.y);
    const float s27 = __fadd_rn(t23.y, t28.y);
    const float s28 = __fadd_rn(-t24.x, t25.x);
    const float s29 = __fadd_rn(-t24.x, -t25.x);
    const float s30 = __fadd_rn(-t24.y, t25.y);
    const float s31 = __fadd_rn(-t24.y, -t25.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// inverse column pass, inputs u < 12 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 20 pair additions and 32 scalar additions
struct InvColT12 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t12 = __fadd2_rn(w[0], w[8]);
    const float2 t13 = sub2(w[0], w[8]);
    const float2 t14 = __fadd2_rn(w[1], w[5]);
    const float2 t15 = sub2(w[1], w[5]);
    const float2 t16 = __fadd2_rn(t12, w[4]);
    const float2 t17 = sub2(w[4], t12);
    const float2 t18 = sub2(w[3], t14);
    const float2 t19 = sub2(w[11], t15);
    const float2 t20 = __fadd2_rn(t15, w[11]);
    const float2 t21 = __fadd2_rn(t14, w[3]);
    const float2 t22 = __fadd2_rn(t16, w[2]);
    const float2 t23 = sub2(w[10], t13);
    const float2 t24 = __fadd2_rn(t13, w[6]);
    const float2 t25 = sub2(w[6], t13);
    const float2 t26 = __fadd2_rn(t13, w[10]);
    const float2 t27 = sub2(w[2], t16);
    const float2 t28 = sub2(w[7], t18);
    const float2 t29 = sub2(w[9], t20);
    const float2 t30 = __fadd2_rn(t20, w[9]);
    const float2 t31 = __fadd2_rn(t18, w[7]);
    const float s0 = __fadd_rn(t21.x, t22.x);
    const float s1 = __fadd_rn(-t21.x, t22.x);
    const float s2 = __fadd_rn(t21.y, t22.y);
    const float s3 = __fadd_rn(-t21.y, t22.y);
    const float s4 = __fadd_rn(-t23.x, t21.x);
    const float s5 = __fadd_rn(-t21.x, -t23.x);
    const float s6 = __fadd_rn(-t23.y, t21.y);
    const float s7 = __fadd_rn(-t21.y, -t23.y);
    const float s8 = __fadd_rn(-t25.x, -t29.x);
    const float s9 = __fadd_rn(-t25.x, t29.x);
    const float s10 = __fadd_rn(-t25.y, -t29.y);
    const float s11 = __fadd_rn(-t25.y, t29.y);
    const float s12 = __fadd_rn(-t17.x, t30.x);
    const float s13 = __fadd_rn(-t17.x, -t30.x);
    const float s14 = __fadd_rn(-t17.y, t30.y);
    const float s15 = __fadd_rn(-t17.y, -t30.y);
    const float s16 = __fadd_rn(-t17.x, -t19.x);
    const float s17 = __fadd_rn(-t17.x, t19.x);
    const float s18 = __fadd_rn(-t17.y, -t19.y);
    const float s19 = __fadd_rn(-t17.y, t19.y);
    const float s20 = __fadd_rn(-t19.x, t24.x);
    const float s21 = __fadd_rn(t19.x, t24.x);
    const float s22 = __fadd_rn(-t19.y, t24.y);
    const float s23 = __fadd_rn(t19.y, t24.y);
    const float s24 = __fadd_rn(-t31.x, t26.x);
    const float s25 = __fadd_rn(t26.x, t31.x);
    const float s26 = __fadd_rn(-t31.y, t26.y);
    const float s27 = __fadd_rn(t26.y, t31.y);
    const float s28 = __fadd_rn(-t27.x, t28.x);
    const float s29 = __fadd_rn(-t27.x, -t28.x);
    const float s30 = __fadd_rn(-t27.y, t28.y);
    const float s31 = __fadd_rn(-t27.y, -t28.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// inverse column pass, inputs u < 13 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 22 pair additions and 32 scalar additions
struct InvColT13 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t13 = __fadd2_rn(w[0], w[8]);
    const float2 t14 = sub2(w[0], w[8]);
    const float2 t15 = __fadd2_rn(w[1], w[5]);
    const float2 t16 = sub2(w[1], w[5]);
    const float2 t17 = __fadd2_rn(t13, w[4]);
    const float2 t18 = sub2(w[12], t14);
    const float2 t19 = __fadd2_rn(t14, w[12]);
    const float2 t20 = sub2(w[4], t13);
    const float2 t21 = sub2(w[3], t15);
    const float2 t22 = sub2(w[11], t16);
    const float2 t23 = __fadd2_rn(t16, w[11]);
    const float2 t24 = __fadd2_rn(t15, w[3]);
    const float2 t25 = __fadd2_rn(t17, w[2]);
    const float2 t26 = __fadd2_rn(t18, w[10]);
    const float2 t27 = __fadd2_rn(t19, w[6]);
    const float2 t28 = sub2(w[6], t19);
    const float2 t29 = sub2(w[10], t18);
    const float2 t30 = sub2(w[2], t17);
    const float2 t31 = sub2(w[7], t21);
    const float2 t32 = sub2(w[9], t23);
    const float2 t33 = __fadd2_rn(t23, w[9]);
    const float2 t34 = __fadd2_rn(t21, w[7]);
    const float s0 = __fadd_rn(t24.x, t25.x);
    const float s1 = __fadd_rn(-t24.x, t25.x);
    const float s2 = __fadd_rn(t24.y, t25.y);
    const float s3 = __fadd_rn(-t24.y, t25.y);
    const float s4 = __fadd_rn(-t26.x, t24.x);
    const float s5 = __fadd_rn(-t24.x, -t26.x);
    const float s6 = __fadd_rn(-t26.y, t24.y);
    const float s7 = __fadd_rn(-t24.y, -t26.y);
    const float s8 = __fadd_rn(-t28.x, -t32.x);
    const float s9 = __fadd_rn(-t28.x, t32.x);
    const float s10 = __fadd_rn(-t28.y, -t32.y);
    const float s11 = __fadd_rn(-t28.y, t32.y);
    const float s12 = __fadd_rn(-t20.x, t33.x);
    const float s13 = __fadd_rn(-t20.x, -t33.x);
    const float s14 = __fadd_rn(-t20.y, t33.y);
    const float s15 = __fadd_rn(-t20.y, -t33.y);
    const float s16 = __fadd_rn(-t20.x, -t22.x);
    const float s17 = __fadd_rn(-t20.x, t22.x);
    const float s18 = __fadd_rn(-t20.y, -t22.y);
    const float s19 = __fadd_rn(-t20.y, t22.y);
    const float s20 = __fadd_rn(-t22.x, t27.x);
    const float s21 = __fadd_rn(t22.x, t27.x);
    const float s22 = __fadd_rn(-t22.y, t27.y);
    const float s23 = __fadd_rn(t22.y, t27.y);
    const float s24 = __fadd_rn(-t34.x, t29.x);
    const float s25 = __fadd_rn(t29.x, t34.x);
    const float s26 = __fadd_rn(-t34.y, t29.y);
    const float s27 = __fadd_rn(t29.y, t34.y);
    const float s28 = __fadd_rn(-t30.x, t31.x);
    const float s29 = __fadd_rn(-t30.x, -t31.x);
    const float s30 = __fadd_rn(-t30.y, t31.y);
    const float s31 = __fadd_rn(-t30.y, -t31.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// inverse column pass, inputs u < 14 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 24 pair additions and 32 scalar additions
struct InvColT14 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t14 = __fadd2_rn(w[0], w[8]);
    const float2 t15 = sub2(w[0], w[8]);
    const float2 t16 = __fadd2_rn(w[1], w[5]);
    const float2 t17 = sub2(w[1], w[5]);
    const float2 t18 = __fadd2_rn(t14, w[4]);
    const float2 t19 = sub2(w[12], t15);
    const float2 t20 = __fadd2_rn(t15, w[12]);
    const float2 t21 = sub2(w[4], t14);
    const float2 t22 = sub2(w[3], t16);
    const float2 t23 = sub2(w[11], t17);
    const float2 t24 = __fadd2_rn(t17, w[11]);
    const float2 t25 = __fadd2_rn(t16, w[3]);
    const float2 t26 = __fadd2_rn(t18, w[2]);
    const float2 t27 = __fadd2_rn(t19, w[10]);
    const float2 t28 = __fadd2_rn(t20, w[6]);
    const float2 t29 = sub2(w[6], t20);
    const float2 t30 = sub2(w[10], t19);
    const float2 t31 = sub2(w[2], t18);
    const float2 t32 = sub2(w[7], t22);
    const float2 t33 = sub2(w[13], t25);
    const float2 t34 = sub2(w[9], t24);
    const float2 t35 = __fadd2_rn(t24, w[9]);
    const float2 t36 = __fadd2_rn(t25, w[13]);
    const float2 t37 = __fadd2_rn(t22, w[7]);
    const float s0 = __fadd_rn(t26.x, t36.x);
    const float s1 = __fadd_rn(-t36.x, t26.x);
    const float s2 = __fadd_rn(t26.y, t36.y);
    const float s3 = __fadd_rn(-t36.y, t26.y);
    const float s4 = __fadd_rn(-t27.x, -t33.x);
    const float s5 = __fadd_rn(-t27.x, t33.x);
    const float s6 = __fadd_rn(-t27.y, -t33.y);
    const float s7 = __fadd_rn(-t27.y, t33.y);
    const float s8 = __fadd_rn(-t29.x, -t34.x);
    const float s9 = __fadd_rn(-t29.x, t34.x);
    const float s10 = __fadd_rn(-t29.y, -t34.y);
    const float s11 = __fadd_rn(-t29.y, t34.y);
    const float s12 = __fadd_rn(-t21.x, t35.x);
    const float s13 = __fadd_rn(-t21.x, -t35.x);
    const float s14 = __fadd_rn(-t21.y, t35.y);
    const float s15 = __fadd_rn(-t21.y, -t35.y);
    const float s16 = __fadd_rn(-t21.x, -t23.x);
    const float s17 = __fadd_rn(-t21.x, t23.x);
    const float s18 = __fadd_rn(-t21.y, -t23.y);
    const float s19 = __fadd_rn(-t21.y, t23.y);
    const float s20 = __fadd_rn(-t23.x, t28.x);
    const float s21 = __fadd_rn(t23.x, t28.x);
    const float s22 = __fadd_rn(-t23.y, t28.y);
    const float s23 = __fadd_rn(t23.y, t28.y);
    const float s24 = __fadd_rn(-t37.x, t30.x);
    const float s25 = __fadd_rn(t30.x, t37.x);
    const float s26 = __fadd_rn(-t37.y, t30.y);
    const float s27 = __fadd_rn(t30.y, t37.y);
    const float s28 = __fadd_rn(-t31.x, t32.x);
    const float s29 = __fadd_rn(-t31.x, -t32.x);
    const float s30 = __fadd_rn(-t31.y, t32.y);
    const float s31 = __fadd_rn(-t31.y, -t32.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// inverse column pass, inputs u < 15 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 26 pair additions and 32 scalar additions
struct InvColT15 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t15 = __fadd2_rn(w[0], w[8]);
    const float2 t16 = sub2(w[0], w[8]);
    const float2 t17 = __fadd2_rn(w[1], w[5]);
    const float2 t18 = sub2(w[1], w[5]);
    const float2 t19 = __fadd2_rn(t15, w[4]);
    const float2 t20 = sub2(w[12], t16);
    const float2 t21 = __fadd2_rn(t16, w[12]);
    const float2 t22 = sub2(w[4], t15);
    const float2 t23 = sub2(w[3], t17);
    const float2 t24 = sub2(w[11], t18);
    const float2 t25 = __fadd2_rn(t18, w[11]);
    const float2 t26 = __fadd2_rn(t17, w[3]);
    const float2 t27 = __fadd2_rn(t19, w[2]);
    const float2 t28 = sub2(w[14], t22);
    const float2 t29 = __fadd2_rn(t20, w[10]);
    const float2 t30 = __fadd2_rn(t21, w[6]);
    const float2 t31 = sub2(w[6], t21);
    const float2 t32 = sub2(w[10], t20);
    const float2 t33 = __fadd2_rn(t22, w[14]);
    const float2 t34 = sub2(w[2], t19);
    const float2 t35 = sub2(w[7], t23);
    const float2 t36 = sub2(w[13], t26);
    const float2 t37 = sub2(w[9], t25);
    const float2 t38 = __fadd2_rn(t25, w[9]);
    const float2 t39 = __fadd2_rn(t26, w[13]);
    const float2 t40 = __fadd2_rn(t23, w[7]);
    const float s0 = __fadd_rn(t27.x, t39.x);
    const float s1 = __fadd_rn(-t39.x, t27.x);
    const float s2 = __fadd_rn(t27.y, t39.y);
    const float s3 = __fadd_rn(-t39.y, t27.y);
    const float s4 = __fadd_rn(-t29.x, -t36.x);
    const float s5 = __fadd_rn(-t29.x, t36.x);
    const float s6 = __fadd_rn(-t29.y, -t36.y);
    const float s7 = __fadd_rn(-t29.y, t36.y);
    const float s8 = __fadd_rn(-t31.x, -t37.x);
    const float s9 = __fadd_rn(-t31.x, t37.x);
    const float s10 = __fadd_rn(-t31.y, -t37.y);
    const float s11 = __fadd_rn(-t31.y, t37.y);
    const float s12 = __fadd_rn(-t33.x, t38.x);
    const float s13 = __fadd_rn(-t33.x, -t38.x);
    const float s14 = __fadd_rn(-t33.y, t38.y);
    const float s15 = __fadd_rn(-t33.y, -t38.y);
    const float s16 = __fadd_rn(-t24.x, t28.x);
    const float s17 = __fadd_rn(t24.x, t28.x);
    const float s18 = __fadd_rn(-t24.y, t28.y);
    const float s19 = __fadd_rn(t24.y, t28.y);
    const float s20 = __fadd_rn(-t24.x, t30.x);
    const float s21 = __fadd_rn(t24.x, t30.x);
    const float s22 = __fadd_rn(-t24.y, t30.y);
    const float s23 = __fadd_rn(t24.y, t30.y);
    const float s24 = __fadd_rn(-t40.x, t32.x);
    const float s25 = __fadd_rn(t32.x, t40.x);
    const float s26 = __fadd_rn(-t40.y, t32.y);
    const float s27 = __fadd_rn(t32.y, t40.y);
    const float s28 = __fadd_rn(-t34.x, t35.x);
    const float s29 = __fadd_rn(-t34.x, -t35.x);
    const float s30 = __fadd_rn(-t34.y, t35.y);
    const float s31 = __fadd_rn(-t34.y, -t35.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// inverse column pass, inputs u < 16 (true values; lanes: columns 2c, 2c+1), with its
// last butterfly (M1) done per lane: Z[i][h] = (z_i, z_(15-i)) of lane h, true values;
// 28 pair additions and 32 scalar additions
struct InvColT16 {
  __device__ static __forceinline__ void run(const float2 (&w)[16], float2 (&Z)[8][2]) {
    const float2 t16 = __fadd2_rn(w[0], w[8]);
    const float2 t17 = sub2(w[0], w[8]);
    const float2 t18 = __fadd2_rn(w[1], w[5]);
    const float2 t19 = sub2(w[1], w[5]);
    const float2 t20 = __fadd2_rn(t16, w[4]);
    const float2 t21 = sub2(w[12], t17);
    const float2 t22 = __fadd2_rn(t17, w[12]);
    const float2 t23 = sub2(w[4], t16);
    const float2 t24 = sub2(w[3], t18);
    const float2 t25 = sub2(w[11], t19);
    const float2 t26 = __fadd2_rn(t19, w[11]);
    const float2 t27 = __fadd2_rn(t18, w[3]);
    const float2 t28 = __fadd2_rn(t20, w[2]);
    const float2 t29 = sub2(w[14], t23);
    const float2 t30 = __fadd2_rn(t21, w[10]);
    const float2 t31 = __fadd2_rn(t22, w[6]);
    const float2 t32 = sub2(w[6], t22);
    const float2 t33 = sub2(w[10], t21);
    const float2 t34 = __fadd2_rn(t23, w[14]);
    const float2 t35 = sub2(w[2], t20);
    const float2 t36 = sub2(w[7], t24);
    const float2 t37 = sub2(w[13], t27);
    const float2 t38 = __fadd2_rn(t25, w[15]);
    const float2 t39 = sub2(w[9], t26);
    const float2 t40 = __fadd2_rn(t26, w[9]);
    const float2 t41 = sub2(w[15], t25);
    const float2 t42 = __fadd2_rn(t27, w[13]);
    const float2 t43 = __fadd2_rn(t24, w[7]);
    const float s0 = __fadd_rn(t28.x, t42.x);
    const float s1 = __fadd_rn(-t42.x, t28.x);
    const float s2 = __fadd_rn(t28.y, t42.y);
    const float s3 = __fadd_rn(-t42.y, t28.y);
    const float s4 = __fadd_rn(-t30.x, -t37.x);
    const float s5 = __fadd_rn(-t30.x, t37.x);
    const float s6 = __fadd_rn(-t30.y, -t37.y);
    const float s7 = __fadd_rn(-t30.y, t37.y);
    const float s8 = __fadd_rn(-t32.x, -t39.x);
    const float s9 = __fadd_rn(-t32.x, t39.x);
    const float s10 = __fadd_rn(-t32.y, -t39.y);
    const float s11 = __fadd_rn(-t32.y, t39.y);
    const float s12 = __fadd_rn(-t34.x, t40.x);
    const float s13 = __fadd_rn(-t34.x, -t40.x);
    const float s14 = __fadd_rn(-t34.y, t40.y);
    const float s15 = __fadd_rn(-t34.y, -t40.y);
    const float s16 = __fadd_rn(-t38.x, t29.x);
    const float s17 = __fadd_rn(t29.x, t38.x);
    const float s18 = __fadd_rn(-t38.y, t29.y);
    const float s19 = __fadd_rn(t29.y, t38.y);
    const float s20 = __fadd_rn(t31.x, t41.x);
    const float s21 = __fadd_rn(-t41.x, t31.x);
    const float s22 = __fadd_rn(t31.y, t41.y);
    const float s23 = __fadd_rn(-t41.y, t31.y);
    const float s24 = __fadd_rn(-t43.x, t33.x);
    const float s25 = __fadd_rn(t33.x, t43.x);
    const float s26 = __fadd_rn(-t43.y, t33.y);
    const float s27 = __fadd_rn(t33.y, t43.y);
    const float s28 = __fadd_rn(-t35.x, t36.x);
    const float s29 = __fadd_rn(-t35.x, -t36.x);
    const float s30 = __fadd_rn(-t35.y, t36.y);
    const float s31 = __fadd_rn(-t35.y, -t36.y);
    Z[0][0] = make_float2(s0, s1);
    Z[0][1] = make_float2(s2, s3);
    Z[1][0] = make_float2(s4, s5);
    Z[1][1] = make_float2(s6, s7);
    Z[2][0] = make_float2(s8, s9);
    Z[2][1] = make_float2(s10, s11);
    Z[3][0] = make_float2(s12, s13);
    Z[3][1] = make_float2(s14, s15);
    Z[4][0] = make_float2(s16, s17);
    Z[4][1] = make_float2(s18, s19);
    Z[5][0] = make_float2(s20, s21);
    Z[5][1] = make_float2(s22, s23);
    Z[6][0] = make_float2(s24, s25);
    Z[6][1] = make_float2(s26, s27);
    Z[7][0] = make_float2(s28, s29);
    Z[7][1] = make_float2(s30, s31);
  }
};

// the column-pass networks of a column pair keeping rows u < H
template <int H>
struct ColNets;
template <>
struct ColNets<1> {
  using FC = FwdColM1;
  using IC = InvColT1;
};
template <>
struct ColNets<2> {
  using FC = FwdColM2;
  using IC = InvColT2;
};
template <>
struct ColNets<3> {
  using FC = FwdColM3;
  using IC = InvColT3;
};
template <>
struct ColNets<4> {
  using FC = FwdColM4;
  using IC = InvColT4;
};
template <>
struct ColNets<5> {
  using FC = FwdColM5;
  using IC = InvColT5;
};
template <>
struct ColNets<6> {
  using FC = FwdColM6;
  using IC = InvColT6;
};
template <>
struct ColNets<7> {
  using FC = FwdColM7;
  using IC = InvColT7;
};
template <>
struct ColNets<8> {
  using FC = FwdColM8;
  using IC = InvColT8;
};
template <>
struct ColNets<9> {
  using FC = FwdColM9;
  using IC = InvColT9;
};
template <>
struct ColNets<10> {
  using FC = FwdColM10;
  using IC = InvColT10;
};
template <>
struct ColNets<11> {
  using FC = FwdColM11;
  using IC = InvColT11;
};
template <>
struct ColNets<12> {
  using FC = FwdColM12;
  using IC = InvColT12;
};
template <>
struct ColNets<13> {
  using FC = FwdColM13;
  using IC = InvColT13;
};
template <>
struct ColNets<14> {
  using FC = FwdColM14;
  using IC = InvColT14;
};
template <>
struct ColNets<15> {
  using FC = FwdColM15;
  using IC = InvColT15;
};
template <>
struct ColNets<16> {
  using FC = FwdColM16;
  using IC = InvColT16;
};

// T8 on one half row of both lanes, outputs v < 1: R[v] = sign[v] * (T8 x)[v];
// 7 pair additions
struct FwdRow8T1 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfffeu, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[1]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t20 = __fadd2_rn(t16, t17);
    R[0] = t20;
  }
};

// T8 on one half row of both lanes, outputs v < 2: R[v] = sign[v] * (T8 x)[v];
// 8 pair additions
struct FwdRow8T2 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfffcu, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[2]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t20 = __fadd2_rn(t16, t17);
    R[0] = t20;
    R[1] = t15;
  }
};

// T8 on one half row of both lanes, outputs v < 3: R[v] = sign[v] * (T8 x)[v];
// 9 pair additions
struct FwdRow8T3 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfff8u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[3]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    R[0] = t20;
    R[1] = t15;
    R[2] = t19;
  }
};

// T8 on one half row of both lanes, outputs v < 4: R[v] = sign[v] * (T8 x)[v];
// 10 pair additions
struct FwdRow8T4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xfff0u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[4]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t11 = sub2(X[2], X[5]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    R[0] = t20;
    R[1] = t15;
    R[2] = t19;
    R[3] = t11;
  }
};

// T8 on one half row of both lanes, outputs v < 5: R[v] = sign[v] * (T8 x)[v];
// 11 pair additions
struct FwdRow8T5 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xffe0u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[5]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t11 = sub2(X[2], X[5]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    R[0] = t20;
    R[1] = t15;
    R[2] = t19;
    R[3] = t11;
    R[4] = t21;
  }
};

// T8 on one half row of both lanes, outputs v < 6: R[v] = sign[v] * (T8 x)[v];
// 12 pair additions
struct FwdRow8T6 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0028u, 0xffc0u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[6]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t11 = sub2(X[2], X[5]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t13 = sub2(X[1], X[6]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    R[0] = t20;
    R[1] = t15;
    R[2] = t19;
    R[3] = t11;
    R[4] = t21;
    R[5] = t13;
  }
};

// T8 on one half row of both lanes, outputs v < 7: R[v] = sign[v] * (T8 x)[v];
// 13 pair additions
struct FwdRow8T7 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0068u, 0xff80u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[7]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t11 = sub2(X[2], X[5]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t13 = sub2(X[1], X[6]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t18 = sub2(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    R[0] = t20;
    R[1] = t15;
    R[2] = t19;
    R[3] = t11;
    R[4] = t21;
    R[5] = t13;
    R[6] = t18;
  }
};

// T8 on one half row of both lanes, outputs v < 8: R[v] = sign[v] * (T8 x)[v];
// 14 pair additions
struct FwdRow8T8 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x00e8u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[8], float2 (&R)[8]) {
    const float2 t8 = __fadd2_rn(X[0], X[7]);
    const float2 t9 = sub2(X[3], X[4]);
    const float2 t10 = __fadd2_rn(X[1], X[6]);
    const float2 t11 = sub2(X[2], X[5]);
    const float2 t12 = __fadd2_rn(X[2], X[5]);
    const float2 t13 = sub2(X[1], X[6]);
    const float2 t14 = __fadd2_rn(X[3], X[4]);
    const float2 t15 = sub2(X[0], X[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t18 = sub2(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    R[0] = t20;
    R[1] = t15;
    R[2] = t19;
    R[3] = t11;
    R[4] = t21;
    R[5] = t13;
    R[6] = t18;
    R[7] = t9;
  }
};

// T8 down a column of the eight row pairs, outputs u < 1: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 7 pair additions
struct FwdCol8M1 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfffeu, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[1]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t20 = __fadd2_rn(t16, t17);
    n[0] = t20;
  }
};

// T8 down a column of the eight row pairs, outputs u < 2: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 8 pair additions
struct FwdCol8M2 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfffcu, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[2]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t20 = __fadd2_rn(t16, t17);
    n[0] = t20;
    n[1] = t15;
  }
};

// T8 down a column of the eight row pairs, outputs u < 3: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 9 pair additions
struct FwdCol8M3 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xfff8u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[3]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    n[0] = t20;
    n[1] = t15;
    n[2] = t19;
  }
};

// T8 down a column of the eight row pairs, outputs u < 4: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 10 pair additions
struct FwdCol8M4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xfff0u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[4]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t11 = sub2(a[2], a[5]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    n[0] = t20;
    n[1] = t15;
    n[2] = t19;
    n[3] = t11;
  }
};

// T8 down a column of the eight row pairs, outputs u < 5: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 11 pair additions
struct FwdCol8M5 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xffe0u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[5]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t11 = sub2(a[2], a[5]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    n[0] = t20;
    n[1] = t15;
    n[2] = t19;
    n[3] = t11;
    n[4] = t21;
  }
};

// T8 down a column of the eight row pairs, outputs u < 6: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 12 pair additions
struct FwdCol8M6 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0028u, 0xffc0u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[6]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t11 = sub2(a[2], a[5]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t13 = sub2(a[1], a[6]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    n[0] = t20;
    n[1] = t15;
    n[2] = t19;
    n[3] = t11;
    n[4] = t21;
    n[5] = t13;
  }
};

// T8 down a column of the eight row pairs, outputs u < 7: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 13 pair additions
struct FwdCol8M7 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0068u, 0xff80u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[7]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t11 = sub2(a[2], a[5]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t13 = sub2(a[1], a[6]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t18 = sub2(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    n[0] = t20;
    n[1] = t15;
    n[2] = t19;
    n[3] = t11;
    n[4] = t21;
    n[5] = t13;
    n[6] = t18;
  }
};

// T8 down a column of the eight row pairs, outputs u < 8: n[u] = sign[u] * (T8 a)[u]
// per lane (lane y: odd u negated, see the row-pair note); 14 pair additions
struct FwdCol8M8 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x00e8u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&a)[8], float2 (&n)[8]) {
    const float2 t8 = __fadd2_rn(a[0], a[7]);
    const float2 t9 = sub2(a[3], a[4]);
    const float2 t10 = __fadd2_rn(a[1], a[6]);
    const float2 t11 = sub2(a[2], a[5]);
    const float2 t12 = __fadd2_rn(a[2], a[5]);
    const float2 t13 = sub2(a[1], a[6]);
    const float2 t14 = __fadd2_rn(a[3], a[4]);
    const float2 t15 = sub2(a[0], a[7]);
    const float2 t16 = __fadd2_rn(t8, t14);
    const float2 t17 = __fadd2_rn(t10, t12);
    const float2 t18 = sub2(t10, t12);
    const float2 t19 = sub2(t8, t14);
    const float2 t20 = __fadd2_rn(t16, t17);
    const float2 t21 = sub2(t16, t17);
    n[0] = t20;
    n[1] = t15;
    n[2] = t19;
    n[3] = t11;
    n[4] = t21;
    n[5] = t13;
    n[6] = t18;
    n[7] = t9;
  }
};

// T8^t down a column, inputs u < 1: z[m] = (T8^t w)[m] per lane, true values; 0 pair additions
struct InvCol8T1 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    z[0] = w[0];
    z[1] = w[0];
    z[2] = w[0];
    z[3] = w[0];
    z[4] = w[0];
    z[5] = w[0];
    z[6] = w[0];
    z[7] = w[0];
  }
};

// T8^t down a column, inputs u < 2: z[m] = (T8^t w)[m] per lane, true values; 2 pair additions
struct InvCol8T2 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t2 = __fadd2_rn(w[0], w[1]);
    const float2 t3 = sub2(w[0], w[1]);
    z[0] = t2;
    z[1] = w[0];
    z[2] = w[0];
    z[3] = w[0];
    z[4] = w[0];
    z[5] = w[0];
    z[6] = w[0];
    z[7] = t3;
  }
};

// T8^t down a column, inputs u < 3: z[m] = (T8^t w)[m] per lane, true values; 4 pair additions
struct InvCol8T3 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t3 = __fadd2_rn(w[0], w[2]);
    const float2 t4 = sub2(w[0], w[2]);
    const float2 t5 = __fadd2_rn(t3, w[1]);
    const float2 t6 = sub2(t3, w[1]);
    z[0] = t5;
    z[1] = w[0];
    z[2] = w[0];
    z[3] = t4;
    z[4] = t4;
    z[5] = w[0];
    z[6] = w[0];
    z[7] = t6;
  }
};

// T8^t down a column, inputs u < 4: z[m] = (T8^t w)[m] per lane, true values; 6 pair additions
struct InvCol8T4 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t4 = __fadd2_rn(w[0], w[2]);
    const float2 t5 = sub2(w[0], w[2]);
    const float2 t6 = __fadd2_rn(t4, w[1]);
    const float2 t7 = __fadd2_rn(w[0], w[3]);
    const float2 t8 = sub2(w[0], w[3]);
    const float2 t9 = sub2(t4, w[1]);
    z[0] = t6;
    z[1] = w[0];
    z[2] = t8;
    z[3] = t5;
    z[4] = t5;
    z[5] = t7;
    z[6] = w[0];
    z[7] = t9;
  }
};

// T8^t down a column, inputs u < 5: z[m] = (T8^t w)[m] per lane, true values; 8 pair additions
struct InvCol8T5 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t5 = __fadd2_rn(w[0], w[4]);
    const float2 t6 = sub2(w[0], w[4]);
    const float2 t7 = __fadd2_rn(t5, w[2]);
    const float2 t8 = sub2(t5, w[2]);
    const float2 t9 = __fadd2_rn(t7, w[1]);
    const float2 t10 = __fadd2_rn(t6, w[3]);
    const float2 t11 = sub2(t6, w[3]);
    const float2 t12 = sub2(t7, w[1]);
    z[0] = t9;
    z[1] = t6;
    z[2] = t11;
    z[3] = t8;
    z[4] = t8;
    z[5] = t10;
    z[6] = t6;
    z[7] = t12;
  }
};

// T8^t down a column, inputs u < 6: z[m] = (T8^t w)[m] per lane, true values; 10 pair additions
struct InvCol8T6 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t6 = __fadd2_rn(w[0], w[4]);
    const float2 t7 = sub2(w[0], w[4]);
    const float2 t8 = __fadd2_rn(t6, w[2]);
    const float2 t9 = sub2(t6, w[2]);
    const float2 t10 = __fadd2_rn(t8, w[1]);
    const float2 t11 = sub2(t7, w[5]);
    const float2 t12 = __fadd2_rn(t7, w[3]);
    const float2 t13 = sub2(t7, w[3]);
    const float2 t14 = __fadd2_rn(t7, w[5]);
    const float2 t15 = sub2(t8, w[1]);
    z[0] = t10;
    z[1] = t11;
    z[2] = t13;
    z[3] = t9;
    z[4] = t9;
    z[5] = t12;
    z[6] = t14;
    z[7] = t15;
  }
};

// T8^t down a column, inputs u < 7: z[m] = (T8^t w)[m] per lane, true values; 12 pair additions
struct InvCol8T7 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t7 = __fadd2_rn(w[0], w[4]);
    const float2 t8 = sub2(w[0], w[4]);
    const float2 t9 = __fadd2_rn(t7, w[2]);
    const float2 t10 = sub2(t8, w[6]);
    const float2 t11 = __fadd2_rn(t8, w[6]);
    const float2 t12 = sub2(t7, w[2]);
    const float2 t13 = __fadd2_rn(t9, w[1]);
    const float2 t14 = sub2(t10, w[5]);
    const float2 t15 = __fadd2_rn(t11, w[3]);
    const float2 t16 = sub2(t11, w[3]);
    const float2 t17 = __fadd2_rn(t10, w[5]);
    const float2 t18 = sub2(t9, w[1]);
    z[0] = t13;
    z[1] = t14;
    z[2] = t16;
    z[3] = t12;
    z[4] = t12;
    z[5] = t15;
    z[6] = t17;
    z[7] = t18;
  }
};

// T8^t down a column, inputs u < 8: z[m] = (T8^t w)[m] per lane, true values; 14 pair additions
struct InvCol8T8 {
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t8 = __fadd2_rn(w[0], w[4]);
    const float2 t9 = sub2(w[0], w[4]);
    const float2 t10 = __fadd2_rn(t8, w[2]);
    const float2 t11 = sub2(t9, w[6]);
    const float2 t12 = __fadd2_rn(t9, w[6]);
    const float2 t13 = sub2(t8, w[2]);
    const float2 t14 = __fadd2_rn(t10, w[1]);
    const float2 t15 = __fadd2_rn(t13, w[7]);
    const float2 t16 = sub2(t11, w[5]);
    const float2 t17 = __fadd2_rn(t12, w[3]);
    const float2 t18 = sub2(t12, w[3]);
    const float2 t19 = __fadd2_rn(t11, w[5]);
    const float2 t20 = sub2(t13, w[7]);
    const float2 t21 = sub2(t10, w[1]);
    z[0] = t14;
    z[1] = t16;
    z[2] = t18;
    z[3] = t20;
    z[4] = t15;
    z[5] = t17;
    z[6] = t19;
    z[7] = t21;
  }
};

// T8^t on a half row, inputs v < 1: z[j] = sign[j] * (T8^t w)[j]; 0 pair additions
struct InvRow8T1 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    z[0] = w[0];
    z[1] = w[0];
    z[2] = w[0];
    z[3] = w[0];
    z[4] = w[0];
    z[5] = w[0];
    z[6] = w[0];
    z[7] = w[0];
  }
};

// T8^t on a half row, inputs v < 2: z[j] = sign[j] * (T8^t w)[j]; 2 pair additions
struct InvRow8T2 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t2 = __fadd2_rn(w[0], w[1]);
    const float2 t3 = sub2(w[0], w[1]);
    z[0] = t2;
    z[1] = w[0];
    z[2] = w[0];
    z[3] = w[0];
    z[4] = w[0];
    z[5] = w[0];
    z[6] = w[0];
    z[7] = t3;
  }
};

// T8^t on a half row, inputs v < 3: z[j] = sign[j] * (T8^t w)[j]; 4 pair additions
struct InvRow8T3 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t3 = __fadd2_rn(w[0], w[2]);
    const float2 t4 = sub2(w[0], w[2]);
    const float2 t5 = __fadd2_rn(t3, w[1]);
    const float2 t6 = sub2(t3, w[1]);
    z[0] = t5;
    z[1] = w[0];
    z[2] = w[0];
    z[3] = t4;
    z[4] = t4;
    z[5] = w[0];
    z[6] = w[0];
    z[7] = t6;
  }
};

// T8^t on a half row, inputs v < 4: z[j] = sign[j] * (T8^t w)[j]; 6 pair additions
struct InvRow8T4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t4 = __fadd2_rn(w[0], w[2]);
    const float2 t5 = sub2(w[0], w[2]);
    const float2 t6 = __fadd2_rn(t4, w[1]);
    const float2 t7 = __fadd2_rn(w[0], w[3]);
    const float2 t8 = sub2(w[0], w[3]);
    const float2 t9 = sub2(t4, w[1]);
    z[0] = t6;
    z[1] = w[0];
    z[2] = t8;
    z[3] = t5;
    z[4] = t5;
    z[5] = t7;
    z[6] = w[0];
    z[7] = t9;
  }
};

// T8^t on a half row, inputs v < 5: z[j] = sign[j] * (T8^t w)[j]; 8 pair additions
struct InvRow8T5 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t5 = __fadd2_rn(w[0], w[4]);
    const float2 t6 = sub2(w[0], w[4]);
    const float2 t7 = __fadd2_rn(t5, w[2]);
    const float2 t8 = sub2(t5, w[2]);
    const float2 t9 = __fadd2_rn(t7, w[1]);
    const float2 t10 = __fadd2_rn(t6, w[3]);
    const float2 t11 = sub2(t6, w[3]);
    const float2 t12 = sub2(t7, w[1]);
    z[0] = t9;
    z[1] = t6;
    z[2] = t11;
    z[3] = t8;
    z[4] = t8;
    z[5] = t10;
    z[6] = t6;
    z[7] = t12;
  }
};

// T8^t on a half row, inputs v < 6: z[j] = sign[j] * (T8^t w)[j]; 10 pair additions
struct InvRow8T6 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t6 = __fadd2_rn(w[0], w[4]);
    const float2 t7 = sub2(w[0], w[4]);
    const float2 t8 = __fadd2_rn(t6, w[2]);
    const float2 t9 = sub2(t6, w[2]);
    const float2 t10 = __fadd2_rn(t8, w[1]);
    const float2 t11 = sub2(t7, w[5]);
    const float2 t12 = __fadd2_rn(t7, w[3]);
    const float2 t13 = sub2(t7, w[3]);
    const float2 t14 = __fadd2_rn(t7, w[5]);
    const float2 t15 = sub2(t8, w[1]);
    z[0] = t10;
    z[1] = t11;
    z[2] = t13;
    z[3] = t9;
    z[4] = t9;
    z[5] = t12;
    z[6] = t14;
    z[7] = t15;
  }
};

// T8^t on a half row, inputs v < 7: z[j] = sign[j] * (T8^t w)[j]; 12 pair additions
struct InvRow8T7 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t7 = __fadd2_rn(w[0], w[4]);
    const float2 t8 = sub2(w[0], w[4]);
    const float2 t9 = __fadd2_rn(t7, w[2]);
    const float2 t10 = sub2(t8, w[6]);
    const float2 t11 = __fadd2_rn(t8, w[6]);
    const float2 t12 = sub2(t7, w[2]);
    const float2 t13 = __fadd2_rn(t9, w[1]);
    const float2 t14 = sub2(t10, w[5]);
    const float2 t15 = __fadd2_rn(t11, w[3]);
    const float2 t16 = sub2(t11, w[3]);
    const float2 t17 = __fadd2_rn(t10, w[5]);
    const float2 t18 = sub2(t9, w[1]);
    z[0] = t13;
    z[1] = t14;
    z[2] = t16;
    z[3] = t12;
    z[4] = t12;
    z[5] = t15;
    z[6] = t17;
    z[7] = t18;
  }
};

// T8^t on a half row, inputs v < 8: z[j] = sign[j] * (T8^t w)[j]; 14 pair additions
struct InvRow8T8 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0000u, 0xff00u, i); }
  __device__ static __forceinline__ void run(const float2 (&w)[8], float2 (&z)[8]) {
    const float2 t8 = __fadd2_rn(w[0], w[4]);
    const float2 t9 = sub2(w[0], w[4]);
    const float2 t10 = __fadd2_rn(t8, w[2]);
    const float2 t11 = sub2(t9, w[6]);
    const float2 t12 = __fadd2_rn(t9, w[6]);
    const float2 t13 = sub2(t8, w[2]);
    const float2 t14 = __fadd2_rn(t10, w[1]);
    const float2 t15 = __fadd2_rn(t13, w[7]);
    const float2 t16 = sub2(t11, w[5]);
    const float2 t17 = __fadd2_rn(t12, w[3]);
    const float2 t18 = sub2(t12, w[3]);
    const float2 t19 = __fadd2_rn(t11, w[5]);
    const float2 t20 = sub2(t13, w[7]);
    const float2 t21 = sub2(t10, w[1]);
    z[0] = t14;
    z[1] = t16;
    z[2] = t18;
    z[3] = t20;
    z[4] = t15;
    z[5] = t17;
    z[6] = t19;
    z[7] = t21;
  }
};

// T8 itself (rows: frequencies u; columns: samples j), for column passes that
// accumulate T8 x term by term; row u is symmetric for even u, antisymmetric
// for odd u
constexpr int kT8[8][8] = {
    {1, 1, 1, 1, 1, 1, 1, 1},
    {1, 0, 0, 0, 0, 0, 0, -1},
    {1, 0, 0, -1, -1, 0, 0, 1},
    {0, 0, -1, 0, 0, 1, 0, 0},
    {1, -1, -1, 1, 1, -1, -1, 1},
    {0, -1, 0, 0, 0, 0, 1, 0},
    {0, -1, 1, 0, 0, 1, -1, 0},
    {0, 0, 0, -1, 1, 0, 0, 0},
};
// the T8 networks of the mixed tiling codec: a column keeping rows u < H,
// a half row keeping columns v < V
template <int H>
struct Col8Nets;
template <>
struct Col8Nets<1> {
  using FC = FwdCol8M1;
  using IC = InvCol8T1;
};
template <>
struct Col8Nets<2> {
  using FC = FwdCol8M2;
  using IC = InvCol8T2;
};
template <>
struct Col8Nets<3> {
  using FC = FwdCol8M3;
  using IC = InvCol8T3;
};
template <>
struct Col8Nets<4> {
  using FC = FwdCol8M4;
  using IC = InvCol8T4;
};
template <>
struct Col8Nets<5> {
  using FC = FwdCol8M5;
  using IC = InvCol8T5;
};
template <>
struct Col8Nets<6> {
  using FC = FwdCol8M6;
  using IC = InvCol8T6;
};
template <>
struct Col8Nets<7> {
  using FC = FwdCol8M7;
  using IC = InvCol8T7;
};
template <>
struct Col8Nets<8> {
  using FC = FwdCol8M8;
  using IC = InvCol8T8;
};
template <int V>
struct Row8Nets;
template <>
struct Row8Nets<1> {
  using FR = FwdRow8T1;
  using IR = InvRow8T1;
};
template <>
struct Row8Nets<2> {
  using FR = FwdRow8T2;
  using IR = InvRow8T2;
};
template <>
struct Row8Nets<3> {
  using FR = FwdRow8T3;
  using IR = InvRow8T3;
};
template <>
struct Row8Nets<4> {
  using FR = FwdRow8T4;
  using IR = InvRow8T4;
};
template <>
struct Row8Nets<5> {
  using FR = FwdRow8T5;
  using IR = InvRow8T5;
};
template <>
struct Row8Nets<6> {
  using FR = FwdRow8T6;
  using IR = InvRow8T6;
};
template <>
struct Row8Nets<7> {
  using FR = FwdRow8T7;
  using IR = InvRow8T7;
};
template <>
struct Row8Nets<8> {
  using FR = FwdRow8T8;
  using IR = InvRow8T8;
};

// sign of each output of the (unpruned) forward network: row-pass outputs
// are stored unsigned; the column thread folds this sign into its scale.
constexpr unsigned kFwdNegMask = 0xdc48u;
}  // namespace pairnet
}  // namespace tx16
