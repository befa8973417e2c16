// GENERATED by gen_networks.py -- do not edit.  The 44-addition network of
// T = P2 M4 M3 M2 P1 M1 (Sec. 2.2) on float2 pairs, negations folded into the
// additions and pruned to the zonal extents used by the fused codec.
#pragma once
#include <cuda_runtime.h>
namespace tx16 {
namespace pairnet {
__device__ __forceinline__ float2 pm1() { return make_float2(-1.f, -1.f); }
__device__ __forceinline__ float2 pbias() { return make_float2(-16777216.f, -16777216.f); }  // -2^24
// sign of output i encoded as bit masks (negative / known zero)
__host__ __device__ constexpr int sign_of(unsigned neg, unsigned zero, int i) {
  return ((zero >> i) & 1u) ? 0 : (((neg >> i) & 1u) ? -1 : 1);
}

// forward row pass, outputs v < 4: y[v] = sign[v] * (T x)[v]; 16 pair additions after M1
struct FwdRow4 {
  __host__ __device__ static constexpr int sign(int i) { return sign_of(0x0008u, 0xfff0u, i); }
  __device__ static __forceinline__ void run(const float2 (&X)[16], float2 (&y)[16]) {
    const float2 a0 = __fadd2_rn(__fadd2_rn(X[0], pbias()), X[15]);
    const float2 a15 = __ffma2_rn(X[15], pm1(), X[0]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = __ffma2_rn(X[14], pm1(), X[1]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = __ffma2_rn(X[13], pm1(), X[2]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = __ffma2_rn(X[12], pm1(), X[3]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = __ffma2_rn(X[11], pm1(), X[4]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = __ffma2_rn(X[10], pm1(), X[5]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = __ffma2_rn(X[9], pm1(), X[6]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = __ffma2_rn(X[8], pm1(), X[7]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = __ffma2_rn(a7, pm1(), a0);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = __ffma2_rn(t30, pm1(), t24);
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
    const float2 a15 = __ffma2_rn(X[15], pm1(), X[0]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = __ffma2_rn(X[14], pm1(), X[1]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = __ffma2_rn(X[13], pm1(), X[2]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = __ffma2_rn(X[12], pm1(), X[3]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = __ffma2_rn(X[11], pm1(), X[4]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = __ffma2_rn(X[10], pm1(), X[5]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = __ffma2_rn(X[9], pm1(), X[6]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = __ffma2_rn(X[8], pm1(), X[7]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = __ffma2_rn(a7, pm1(), a0);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = __ffma2_rn(t22, pm1(), t16);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = __ffma2_rn(t30, pm1(), t24);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = __ffma2_rn(t37, pm1(), t36);
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
    const float2 a15 = __ffma2_rn(X[15], pm1(), X[0]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = __ffma2_rn(X[14], pm1(), X[1]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = __ffma2_rn(X[13], pm1(), X[2]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = __ffma2_rn(X[12], pm1(), X[3]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = __ffma2_rn(X[11], pm1(), X[4]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = __ffma2_rn(X[10], pm1(), X[5]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = __ffma2_rn(X[9], pm1(), X[6]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = __ffma2_rn(X[8], pm1(), X[7]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t19 = __ffma2_rn(a5, pm1(), a2);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = __ffma2_rn(a7, pm1(), a0);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t31 = __ffma2_rn(a9, pm1(), a8);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = __ffma2_rn(t22, pm1(), t16);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = __ffma2_rn(t30, pm1(), t24);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = __ffma2_rn(t37, pm1(), t36);
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
    const float2 a15 = __ffma2_rn(X[15], pm1(), X[0]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = __ffma2_rn(X[14], pm1(), X[1]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = __ffma2_rn(X[13], pm1(), X[2]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = __ffma2_rn(X[12], pm1(), X[3]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = __ffma2_rn(X[11], pm1(), X[4]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = __ffma2_rn(X[10], pm1(), X[5]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = __ffma2_rn(X[9], pm1(), X[6]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = __ffma2_rn(X[8], pm1(), X[7]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t19 = __ffma2_rn(a5, pm1(), a2);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = __ffma2_rn(a7, pm1(), a0);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t27 = __ffma2_rn(a13, pm1(), a12);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t31 = __ffma2_rn(a9, pm1(), a8);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t35 = __ffma2_rn(t22, pm1(), t16);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t39 = __ffma2_rn(t30, pm1(), t24);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = __ffma2_rn(t33, pm1(), t32);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = __ffma2_rn(t37, pm1(), t36);
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
    const float2 a15 = __ffma2_rn(X[15], pm1(), X[0]);
    const float2 a1 = __fadd2_rn(__fadd2_rn(X[1], pbias()), X[14]);
    const float2 a14 = __ffma2_rn(X[14], pm1(), X[1]);
    const float2 a2 = __fadd2_rn(__fadd2_rn(X[2], pbias()), X[13]);
    const float2 a13 = __ffma2_rn(X[13], pm1(), X[2]);
    const float2 a3 = __fadd2_rn(__fadd2_rn(X[3], pbias()), X[12]);
    const float2 a12 = __ffma2_rn(X[12], pm1(), X[3]);
    const float2 a4 = __fadd2_rn(__fadd2_rn(X[4], pbias()), X[11]);
    const float2 a11 = __ffma2_rn(X[11], pm1(), X[4]);
    const float2 a5 = __fadd2_rn(__fadd2_rn(X[5], pbias()), X[10]);
    const float2 a10 = __ffma2_rn(X[10], pm1(), X[5]);
    const float2 a6 = __fadd2_rn(__fadd2_rn(X[6], pbias()), X[9]);
    const float2 a9 = __ffma2_rn(X[9], pm1(), X[6]);
    const float2 a7 = __fadd2_rn(__fadd2_rn(X[7], pbias()), X[8]);
    const float2 a8 = __ffma2_rn(X[8], pm1(), X[7]);
    const float2 t16 = __fadd2_rn(a0, a7);
    const float2 t17 = __ffma2_rn(a4, pm1(), a3);
    const float2 t18 = __fadd2_rn(a1, a6);
    const float2 t19 = __ffma2_rn(a5, pm1(), a2);
    const float2 t20 = __fadd2_rn(a2, a5);
    const float2 t21 = __ffma2_rn(a6, pm1(), a1);
    const float2 t22 = __fadd2_rn(a3, a4);
    const float2 t23 = __ffma2_rn(a7, pm1(), a0);
    const float2 t24 = __fadd2_rn(a8, a9);
    const float2 t25 = __ffma2_rn(a14, pm1(), a15);
    const float2 t26 = __fadd2_rn(a11, a10);
    const float2 t27 = __ffma2_rn(a13, pm1(), a12);
    const float2 t28 = __fadd2_rn(a12, a13);
    const float2 t29 = __ffma2_rn(a10, pm1(), a11);
    const float2 t30 = __fadd2_rn(a15, a14);
    const float2 t31 = __ffma2_rn(a9, pm1(), a8);
    const float2 t32 = __fadd2_rn(t16, t22);
    const float2 t33 = __fadd2_rn(t18, t20);
    const float2 t34 = __ffma2_rn(t20, pm1(), t18);
    const float2 t35 = __ffma2_rn(t22, pm1(), t16);
    const float2 t36 = __fadd2_rn(t24, t30);
    const float2 t37 = __fadd2_rn(t26, t28);
    const float2 t38 = __ffma2_rn(t28, pm1(), t26);
    const float2 t39 = __ffma2_rn(t30, pm1(), t24);
    const float2 t40 = __fadd2_rn(t32, t33);
    const float2 t41 = __ffma2_rn(t33, pm1(), t32);
    const float2 t42 = __fadd2_rn(t36, t37);
    const float2 t43 = __ffma2_rn(t37, pm1(), t36);
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
    const float2 t17 = __ffma2_rn(x[8], pm1(), x[7]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = __ffma2_rn(x[9], pm1(), x[6]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = __ffma2_rn(x[10], pm1(), x[5]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = __ffma2_rn(x[11], pm1(), x[4]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = __ffma2_rn(x[12], pm1(), x[3]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = __ffma2_rn(x[13], pm1(), x[2]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = __ffma2_rn(x[14], pm1(), x[1]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = __ffma2_rn(x[15], pm1(), x[0]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = __ffma2_rn(t30, pm1(), t16);
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
    const float2 t17 = __ffma2_rn(x[8], pm1(), x[7]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = __ffma2_rn(x[9], pm1(), x[6]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = __ffma2_rn(x[10], pm1(), x[5]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = __ffma2_rn(x[11], pm1(), x[4]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = __ffma2_rn(x[12], pm1(), x[3]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = __ffma2_rn(x[13], pm1(), x[2]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = __ffma2_rn(x[14], pm1(), x[1]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = __ffma2_rn(x[15], pm1(), x[0]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = __ffma2_rn(t30, pm1(), t16);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = __ffma2_rn(t38, pm1(), t32);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = __ffma2_rn(t46, pm1(), t40);
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
    const float2 t17 = __ffma2_rn(x[8], pm1(), x[7]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = __ffma2_rn(x[9], pm1(), x[6]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = __ffma2_rn(x[10], pm1(), x[5]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = __ffma2_rn(x[11], pm1(), x[4]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = __ffma2_rn(x[12], pm1(), x[3]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = __ffma2_rn(x[13], pm1(), x[2]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = __ffma2_rn(x[14], pm1(), x[1]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = __ffma2_rn(x[15], pm1(), x[0]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = __ffma2_rn(t26, pm1(), t20);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = __ffma2_rn(t30, pm1(), t16);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = __ffma2_rn(t38, pm1(), t32);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = __ffma2_rn(t46, pm1(), t40);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = __ffma2_rn(t53, pm1(), t52);
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
    const float2 t17 = __ffma2_rn(x[8], pm1(), x[7]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = __ffma2_rn(x[9], pm1(), x[6]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = __ffma2_rn(x[10], pm1(), x[5]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = __ffma2_rn(x[11], pm1(), x[4]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = __ffma2_rn(x[12], pm1(), x[3]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = __ffma2_rn(x[13], pm1(), x[2]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = __ffma2_rn(x[14], pm1(), x[1]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = __ffma2_rn(x[15], pm1(), x[0]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = __ffma2_rn(t26, pm1(), t20);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t37 = __ffma2_rn(t28, pm1(), t18);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = __ffma2_rn(t30, pm1(), t16);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t43 = __ffma2_rn(t27, pm1(), t25);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = __ffma2_rn(t19, pm1(), t17);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t51 = __ffma2_rn(t38, pm1(), t32);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t55 = __ffma2_rn(t46, pm1(), t40);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t57 = __ffma2_rn(t49, pm1(), t48);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = __ffma2_rn(t53, pm1(), t52);
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
    const float2 t17 = __ffma2_rn(x[8], pm1(), x[7]);
    const float2 t18 = __fadd2_rn(x[1], x[14]);
    const float2 t19 = __ffma2_rn(x[9], pm1(), x[6]);
    const float2 t20 = __fadd2_rn(x[2], x[13]);
    const float2 t21 = __ffma2_rn(x[10], pm1(), x[5]);
    const float2 t22 = __fadd2_rn(x[3], x[12]);
    const float2 t23 = __ffma2_rn(x[11], pm1(), x[4]);
    const float2 t24 = __fadd2_rn(x[4], x[11]);
    const float2 t25 = __ffma2_rn(x[12], pm1(), x[3]);
    const float2 t26 = __fadd2_rn(x[5], x[10]);
    const float2 t27 = __ffma2_rn(x[13], pm1(), x[2]);
    const float2 t28 = __fadd2_rn(x[6], x[9]);
    const float2 t29 = __ffma2_rn(x[14], pm1(), x[1]);
    const float2 t30 = __fadd2_rn(x[7], x[8]);
    const float2 t31 = __ffma2_rn(x[15], pm1(), x[0]);
    const float2 t32 = __fadd2_rn(t16, t30);
    const float2 t33 = __ffma2_rn(t24, pm1(), t22);
    const float2 t34 = __fadd2_rn(t18, t28);
    const float2 t35 = __ffma2_rn(t26, pm1(), t20);
    const float2 t36 = __fadd2_rn(t20, t26);
    const float2 t37 = __ffma2_rn(t28, pm1(), t18);
    const float2 t38 = __fadd2_rn(t22, t24);
    const float2 t39 = __ffma2_rn(t30, pm1(), t16);
    const float2 t40 = __fadd2_rn(t17, t19);
    const float2 t41 = __ffma2_rn(t29, pm1(), t31);
    const float2 t42 = __fadd2_rn(t23, t21);
    const float2 t43 = __ffma2_rn(t27, pm1(), t25);
    const float2 t44 = __fadd2_rn(t25, t27);
    const float2 t45 = __ffma2_rn(t21, pm1(), t23);
    const float2 t46 = __fadd2_rn(t31, t29);
    const float2 t47 = __ffma2_rn(t19, pm1(), t17);
    const float2 t48 = __fadd2_rn(t32, t38);
    const float2 t49 = __fadd2_rn(t34, t36);
    const float2 t50 = __ffma2_rn(t36, pm1(), t34);
    const float2 t51 = __ffma2_rn(t38, pm1(), t32);
    const float2 t52 = __fadd2_rn(t40, t46);
    const float2 t53 = __fadd2_rn(t42, t44);
    const float2 t54 = __ffma2_rn(t44, pm1(), t42);
    const float2 t55 = __ffma2_rn(t46, pm1(), t40);
    const float2 t56 = __fadd2_rn(t48, t49);
    const float2 t57 = __ffma2_rn(t49, pm1(), t48);
    const float2 t58 = __fadd2_rn(t52, t53);
    const float2 t59 = __ffma2_rn(t53, pm1(), t52);
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
    const float2 t4 = __ffma2_rn(w[2], pm1(), w[0]);
    const float2 t5 = __fadd2_rn(t3, w[1]);
    const float2 t6 = __ffma2_rn(w[1], pm1(), t4);
    const float2 t7 = __fadd2_rn(w[0], w[1]);
    const float2 t8 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t9 = __fadd2_rn(w[0], w[1]);
    const float2 t10 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t11 = __fadd2_rn(w[0], w[1]);
    const float2 t12 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t13 = __fadd2_rn(w[0], w[1]);
    const float2 t14 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t15 = __fadd2_rn(w[0], w[1]);
    const float2 t16 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t17 = __fadd2_rn(w[0], w[1]);
    const float2 t18 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t19 = __fadd2_rn(t4, w[1]);
    const float2 t20 = __ffma2_rn(w[1], pm1(), t3);
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
    const float2 t6 = __ffma2_rn(w[4], pm1(), w[0]);
    const float2 t7 = __fadd2_rn(w[1], w[3]);
    const float2 t8 = __ffma2_rn(w[3], pm1(), w[1]);
    const float2 t9 = __fadd2_rn(t5, w[2]);
    const float2 t10 = __ffma2_rn(w[2], pm1(), t5);
    const float2 t11 = __fadd2_rn(t9, t8);
    const float2 t12 = __ffma2_rn(t7, pm1(), t10);
    const float2 t13 = __fadd2_rn(w[0], t8);
    const float2 t14 = __ffma2_rn(t7, pm1(), w[0]);
    const float2 t15 = __fadd2_rn(w[0], w[1]);
    const float2 t16 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t17 = __fadd2_rn(t6, w[1]);
    const float2 t18 = __ffma2_rn(w[1], pm1(), t6);
    const float2 t19 = __fadd2_rn(t6, w[1]);
    const float2 t20 = __ffma2_rn(w[1], pm1(), t6);
    const float2 t21 = __fadd2_rn(w[0], w[1]);
    const float2 t22 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t23 = __fadd2_rn(w[0], t7);
    const float2 t24 = __ffma2_rn(t8, pm1(), w[0]);
    const float2 t25 = __fadd2_rn(t10, t7);
    const float2 t26 = __ffma2_rn(t8, pm1(), t9);
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
    const float2 t8 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t9 = __fadd2_rn(w[0], w[4]);
    const float2 t10 = __ffma2_rn(w[4], pm1(), w[0]);
    const float2 t11 = __fadd2_rn(t7, w[3]);
    const float2 t12 = __ffma2_rn(w[3], pm1(), t7);
    const float2 t13 = __fadd2_rn(t9, w[2]);
    const float2 t14 = __ffma2_rn(w[6], pm1(), w[0]);
    const float2 t15 = __fadd2_rn(w[0], w[6]);
    const float2 t16 = __ffma2_rn(w[2], pm1(), t9);
    const float2 t17 = __fadd2_rn(t13, t12);
    const float2 t18 = __ffma2_rn(t11, pm1(), t16);
    const float2 t19 = __fadd2_rn(w[0], t12);
    const float2 t20 = __ffma2_rn(t11, pm1(), w[0]);
    const float2 t21 = __fadd2_rn(t15, t8);
    const float2 t22 = __ffma2_rn(t8, pm1(), t14);
    const float2 t23 = __fadd2_rn(t10, t8);
    const float2 t24 = __ffma2_rn(t8, pm1(), t10);
    const float2 t25 = __fadd2_rn(t10, t8);
    const float2 t26 = __ffma2_rn(t8, pm1(), t10);
    const float2 t27 = __fadd2_rn(t14, t8);
    const float2 t28 = __ffma2_rn(t8, pm1(), t15);
    const float2 t29 = __fadd2_rn(w[0], t11);
    const float2 t30 = __ffma2_rn(t12, pm1(), w[0]);
    const float2 t31 = __fadd2_rn(t16, t11);
    const float2 t32 = __ffma2_rn(t12, pm1(), t13);
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
    const float2 t12 = __ffma2_rn(w[8], pm1(), w[0]);
    const float2 t13 = __fadd2_rn(w[1], w[5]);
    const float2 t14 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t15 = __fadd2_rn(t11, w[4]);
    const float2 t16 = __ffma2_rn(w[4], pm1(), t11);
    const float2 t17 = __fadd2_rn(t13, w[3]);
    const float2 t18 = __ffma2_rn(w[3], pm1(), t13);
    const float2 t19 = __fadd2_rn(t15, w[2]);
    const float2 t20 = __fadd2_rn(t12, w[10]);
    const float2 t21 = __ffma2_rn(w[6], pm1(), t12);
    const float2 t22 = __fadd2_rn(t12, w[6]);
    const float2 t23 = __ffma2_rn(w[10], pm1(), t12);
    const float2 t24 = __ffma2_rn(w[2], pm1(), t15);
    const float2 t25 = __fadd2_rn(t17, w[7]);
    const float2 t26 = __ffma2_rn(w[9], pm1(), t14);
    const float2 t27 = __fadd2_rn(t14, w[9]);
    const float2 t28 = __ffma2_rn(w[7], pm1(), t17);
    const float2 t29 = __fadd2_rn(t19, t18);
    const float2 t30 = __ffma2_rn(t25, pm1(), t24);
    const float2 t31 = __fadd2_rn(t20, t18);
    const float2 t32 = __ffma2_rn(t28, pm1(), t23);
    const float2 t33 = __fadd2_rn(t22, t26);
    const float2 t34 = __ffma2_rn(t14, pm1(), t21);
    const float2 t35 = __fadd2_rn(t16, t27);
    const float2 t36 = __ffma2_rn(t14, pm1(), t16);
    const float2 t37 = __fadd2_rn(t16, t14);
    const float2 t38 = __ffma2_rn(t27, pm1(), t16);
    const float2 t39 = __fadd2_rn(t21, t14);
    const float2 t40 = __ffma2_rn(t26, pm1(), t22);
    const float2 t41 = __fadd2_rn(t23, t28);
    const float2 t42 = __ffma2_rn(t18, pm1(), t20);
    const float2 t43 = __fadd2_rn(t24, t25);
    const float2 t44 = __ffma2_rn(t18, pm1(), t19);
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
    const float2 t17 = __ffma2_rn(w[8], pm1(), w[0]);
    const float2 t18 = __fadd2_rn(w[1], w[5]);
    const float2 t19 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t20 = __fadd2_rn(t16, w[4]);
    const float2 t21 = __fadd2_rn(t17, w[12]);
    const float2 t22 = __ffma2_rn(w[12], pm1(), t17);
    const float2 t23 = __ffma2_rn(w[4], pm1(), t16);
    const float2 t24 = __fadd2_rn(t18, w[3]);
    const float2 t25 = __fadd2_rn(t19, w[11]);
    const float2 t26 = __ffma2_rn(w[11], pm1(), t19);
    const float2 t27 = __ffma2_rn(w[3], pm1(), t18);
    const float2 t28 = __fadd2_rn(t20, w[2]);
    const float2 t29 = __ffma2_rn(w[14], pm1(), t23);
    const float2 t30 = __fadd2_rn(t21, w[10]);
    const float2 t31 = __ffma2_rn(w[6], pm1(), t22);
    const float2 t32 = __fadd2_rn(t22, w[6]);
    const float2 t33 = __ffma2_rn(w[10], pm1(), t21);
    const float2 t34 = __fadd2_rn(t23, w[14]);
    const float2 t35 = __ffma2_rn(w[2], pm1(), t20);
    const float2 t36 = __fadd2_rn(t24, w[7]);
    const float2 t37 = __ffma2_rn(w[13], pm1(), t27);
    const float2 t38 = __fadd2_rn(t25, w[15]);
    const float2 t39 = __ffma2_rn(w[9], pm1(), t26);
    const float2 t40 = __fadd2_rn(t26, w[9]);
    const float2 t41 = __ffma2_rn(w[15], pm1(), t25);
    const float2 t42 = __fadd2_rn(t27, w[13]);
    const float2 t43 = __ffma2_rn(w[7], pm1(), t24);
    const float2 t44 = __fadd2_rn(t28, t42);
    const float2 t45 = __ffma2_rn(t36, pm1(), t35);
    const float2 t46 = __fadd2_rn(t30, t37);
    const float2 t47 = __ffma2_rn(t43, pm1(), t33);
    const float2 t48 = __fadd2_rn(t32, t39);
    const float2 t49 = __ffma2_rn(t41, pm1(), t31);
    const float2 t50 = __fadd2_rn(t34, t40);
    const float2 t51 = __ffma2_rn(t38, pm1(), t29);
    const float2 t52 = __fadd2_rn(t29, t38);
    const float2 t53 = __ffma2_rn(t40, pm1(), t34);
    const float2 t54 = __fadd2_rn(t31, t41);
    const float2 t55 = __ffma2_rn(t39, pm1(), t32);
    const float2 t56 = __fadd2_rn(t33, t43);
    const float2 t57 = __ffma2_rn(t37, pm1(), t30);
    const float2 t58 = __fadd2_rn(t35, t36);
    const float2 t59 = __ffma2_rn(t42, pm1(), t28);
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
    const float2 t4 = __ffma2_rn(w[3], pm1(), w[1]);
    const float2 t5 = __fadd2_rn(w[1], w[3]);
    const float2 t6 = __fadd2_rn(w[0], w[2]);
    const float2 t7 = __ffma2_rn(w[2], pm1(), w[0]);
    const float2 t8 = __fadd2_rn(t6, t5);
    const float2 t9 = __ffma2_rn(t4, pm1(), t7);
    const float2 t10 = __fadd2_rn(w[0], t5);
    const float2 t11 = __ffma2_rn(t4, pm1(), w[0]);
    const float2 t12 = __fadd2_rn(w[0], w[1]);
    const float2 t13 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t14 = __fadd2_rn(w[0], w[1]);
    const float2 t15 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t16 = __fadd2_rn(w[0], w[1]);
    const float2 t17 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t18 = __fadd2_rn(w[0], w[1]);
    const float2 t19 = __ffma2_rn(w[1], pm1(), w[0]);
    const float2 t20 = __fadd2_rn(w[0], t4);
    const float2 t21 = __ffma2_rn(t5, pm1(), w[0]);
    const float2 t22 = __fadd2_rn(t7, t4);
    const float2 t23 = __ffma2_rn(t5, pm1(), t6);
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
    const float2 t7 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t8 = __fadd2_rn(w[0], w[4]);
    const float2 t9 = __ffma2_rn(w[4], pm1(), w[0]);
    const float2 t10 = __ffma2_rn(w[3], pm1(), t6);
    const float2 t11 = __fadd2_rn(t6, w[3]);
    const float2 t12 = __fadd2_rn(t8, w[2]);
    const float2 t13 = __ffma2_rn(w[2], pm1(), t8);
    const float2 t14 = __fadd2_rn(t12, t11);
    const float2 t15 = __ffma2_rn(t10, pm1(), t13);
    const float2 t16 = __fadd2_rn(w[0], t11);
    const float2 t17 = __ffma2_rn(t10, pm1(), w[0]);
    const float2 t18 = __fadd2_rn(w[0], t7);
    const float2 t19 = __ffma2_rn(t7, pm1(), w[0]);
    const float2 t20 = __fadd2_rn(t9, t7);
    const float2 t21 = __ffma2_rn(t7, pm1(), t9);
    const float2 t22 = __fadd2_rn(t9, t7);
    const float2 t23 = __ffma2_rn(t7, pm1(), t9);
    const float2 t24 = __fadd2_rn(w[0], t7);
    const float2 t25 = __ffma2_rn(t7, pm1(), w[0]);
    const float2 t26 = __fadd2_rn(w[0], t10);
    const float2 t27 = __ffma2_rn(t11, pm1(), w[0]);
    const float2 t28 = __fadd2_rn(t13, t10);
    const float2 t29 = __ffma2_rn(t11, pm1(), t12);
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
    const float2 t9 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t10 = __fadd2_rn(w[0], w[4]);
    const float2 t11 = __ffma2_rn(w[4], pm1(), w[0]);
    const float2 t12 = __ffma2_rn(w[3], pm1(), t8);
    const float2 t13 = __fadd2_rn(t8, w[3]);
    const float2 t14 = __fadd2_rn(t10, w[2]);
    const float2 t15 = __fadd2_rn(w[0], w[6]);
    const float2 t16 = __ffma2_rn(w[6], pm1(), w[0]);
    const float2 t17 = __ffma2_rn(w[2], pm1(), t10);
    const float2 t18 = __fadd2_rn(t12, w[7]);
    const float2 t19 = __ffma2_rn(w[7], pm1(), t12);
    const float2 t20 = __fadd2_rn(t14, t13);
    const float2 t21 = __ffma2_rn(t18, pm1(), t17);
    const float2 t22 = __fadd2_rn(w[0], t13);
    const float2 t23 = __ffma2_rn(t19, pm1(), w[0]);
    const float2 t24 = __fadd2_rn(t16, t9);
    const float2 t25 = __ffma2_rn(t9, pm1(), t15);
    const float2 t26 = __fadd2_rn(t11, t9);
    const float2 t27 = __ffma2_rn(t9, pm1(), t11);
    const float2 t28 = __fadd2_rn(t11, t9);
    const float2 t29 = __ffma2_rn(t9, pm1(), t11);
    const float2 t30 = __fadd2_rn(t15, t9);
    const float2 t31 = __ffma2_rn(t9, pm1(), t16);
    const float2 t32 = __fadd2_rn(w[0], t19);
    const float2 t33 = __ffma2_rn(t13, pm1(), w[0]);
    const float2 t34 = __fadd2_rn(t17, t18);
    const float2 t35 = __ffma2_rn(t13, pm1(), t14);
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
    const float2 t11 = __ffma2_rn(w[8], pm1(), w[0]);
    const float2 t12 = __fadd2_rn(w[1], w[5]);
    const float2 t13 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t14 = __fadd2_rn(t10, w[4]);
    const float2 t15 = __ffma2_rn(w[4], pm1(), t10);
    const float2 t16 = __ffma2_rn(w[3], pm1(), t12);
    const float2 t17 = __fadd2_rn(t12, w[3]);
    const float2 t18 = __fadd2_rn(t14, w[2]);
    const float2 t19 = __fadd2_rn(t11, w[6]);
    const float2 t20 = __ffma2_rn(w[6], pm1(), t11);
    const float2 t21 = __ffma2_rn(w[2], pm1(), t14);
    const float2 t22 = __fadd2_rn(t16, w[7]);
    const float2 t23 = __ffma2_rn(w[9], pm1(), t13);
    const float2 t24 = __fadd2_rn(t13, w[9]);
    const float2 t25 = __ffma2_rn(w[7], pm1(), t16);
    const float2 t26 = __fadd2_rn(t18, t17);
    const float2 t27 = __ffma2_rn(t22, pm1(), t21);
    const float2 t28 = __fadd2_rn(t11, t17);
    const float2 t29 = __ffma2_rn(t25, pm1(), t11);
    const float2 t30 = __fadd2_rn(t20, t23);
    const float2 t31 = __ffma2_rn(t13, pm1(), t19);
    const float2 t32 = __fadd2_rn(t15, t24);
    const float2 t33 = __ffma2_rn(t13, pm1(), t15);
    const float2 t34 = __fadd2_rn(t15, t13);
    const float2 t35 = __ffma2_rn(t24, pm1(), t15);
    const float2 t36 = __fadd2_rn(t19, t13);
    const float2 t37 = __ffma2_rn(t23, pm1(), t20);
    const float2 t38 = __fadd2_rn(t11, t25);
    const float2 t39 = __ffma2_rn(t17, pm1(), t11);
    const float2 t40 = __fadd2_rn(t21, t22);
    const float2 t41 = __ffma2_rn(t17, pm1(), t18);
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
    const float2 t17 = __ffma2_rn(w[8], pm1(), w[0]);
    const float2 t18 = __fadd2_rn(w[1], w[5]);
    const float2 t19 = __ffma2_rn(w[5], pm1(), w[1]);
    const float2 t20 = __fadd2_rn(t16, w[4]);
    const float2 t21 = __ffma2_rn(w[12], pm1(), t17);
    const float2 t22 = __fadd2_rn(t17, w[12]);
    const float2 t23 = __ffma2_rn(w[4], pm1(), t16);
    const float2 t24 = __ffma2_rn(w[3], pm1(), t18);
    const float2 t25 = __ffma2_rn(w[11], pm1(), t19);
    const float2 t26 = __fadd2_rn(t19, w[11]);
    const float2 t27 = __fadd2_rn(t18, w[3]);
    const float2 t28 = __fadd2_rn(t20, w[2]);
    const float2 t29 = __fadd2_rn(t23, w[14]);
    const float2 t30 = __ffma2_rn(w[10], pm1(), t21);
    const float2 t31 = __fadd2_rn(t22, w[6]);
    const float2 t32 = __ffma2_rn(w[6], pm1(), t22);
    const float2 t33 = __fadd2_rn(t21, w[10]);
    const float2 t34 = __ffma2_rn(w[14], pm1(), t23);
    const float2 t35 = __ffma2_rn(w[2], pm1(), t20);
    const float2 t36 = __fadd2_rn(t24, w[7]);
    const float2 t37 = __ffma2_rn(w[13], pm1(), t27);
    const float2 t38 = __ffma2_rn(w[15], pm1(), t25);
    const float2 t39 = __ffma2_rn(w[9], pm1(), t26);
    const float2 t40 = __fadd2_rn(t26, w[9]);
    const float2 t41 = __fadd2_rn(t25, w[15]);
    const float2 t42 = __fadd2_rn(t27, w[13]);
    const float2 t43 = __ffma2_rn(w[7], pm1(), t24);
    const float2 t44 = __fadd2_rn(t28, t42);
    const float2 t45 = __ffma2_rn(t36, pm1(), t35);
    const float2 t46 = __fadd2_rn(t30, t37);
    const float2 t47 = __ffma2_rn(t43, pm1(), t33);
    const float2 t48 = __fadd2_rn(t32, t39);
    const float2 t49 = __ffma2_rn(t41, pm1(), t31);
    const float2 t50 = __fadd2_rn(t34, t40);
    const float2 t51 = __ffma2_rn(t38, pm1(), t29);
    const float2 t52 = __fadd2_rn(t29, t38);
    const float2 t53 = __ffma2_rn(t40, pm1(), t34);
    const float2 t54 = __fadd2_rn(t31, t41);
    const float2 t55 = __ffma2_rn(t39, pm1(), t32);
    const float2 t56 = __fadd2_rn(t33, t43);
    const float2 t57 = __ffma2_rn(t37, pm1(), t30);
    const float2 t58 = __fadd2_rn(t35, t36);
    const float2 t59 = __ffma2_rn(t42, pm1(), t28);
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

// sign of each output of the (unpruned) forward network: row-pass outputs
// are stored unsigned; the column thread folds this sign into its scale.
constexpr unsigned kFwdNegMask = 0xdc48u;
}  // namespace pairnet
}  // namespace tx16
