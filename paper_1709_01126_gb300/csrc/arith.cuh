// Arithmetic policies for the PCG kernels.
//
// The same kernel templates run in three arithmetics:
//   PF64  native FP64 (one DFMA per multiply-add),
//   PDF   double-float: a value is an unevaluated sum hi + lo of two floats
//         (|lo| <= ulp(hi)/2, about 48 significant bits); every operation
//         runs on the FP32 units with error-free transformations,
//   PF32  single precision (the inner solve of iterative refinement).
// GB300 executes FP32 FMAs at 128 per SM per clock and FP64 FMAs at about
// 2, so PDF is the FP64-class arithmetic that keeps up with HBM.
//
// Double-float building blocks:
//   TwoSum (Knuth), FastTwoSum (Dekker), TwoProd by FMA;
//   DWPlusDW ("accurate" variant) and DWTimesDW with FMA from
//   M. Joldes, J.-M. Muller, V. Popescu, "Tight and rigorous error bounds for
//   basic building blocks of double-word arithmetic", ACM TOMS 44(2), 2017;
//   dot products are accumulated as in T. Ogita, S. Rump, S. Oishi,
//   "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6), 2005 (Dot2).
// The explicit __f*_rn intrinsics keep nvcc from contracting or reordering
// the error-free transformations.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pot3d {

struct dfl {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  float sh, sl, th, tl;
  two_sum(x.h, y.h, sh, sl);
  two_sum(x.l, y.l, th, tl);
  sl = __fadd_rn(sl, th);
  fast_two_sum(sh, sl, sh, sl);
  sl = __fadd_rn(sl, tl);
  dfl z;
  fast_two_sum(sh, sl, z.h, z.l);
  return z;
}

// SloppyDWPlusDW: the relative error bound holds when x and y have the same
// sign; under cancellation the absolute error stays within about 2^-46 of
// |x| + |y|, which is the accuracy an accumulator (x~, r, p~) needs.
__device__ __forceinline__ dfl df_add_sloppy(dfl x, dfl y) {
  float sh, sl;
  two_sum(x.h, y.h, sh, sl);
  sl = __fadd_rn(sl, __fadd_rn(x.l, y.l));
  dfl z;
  fast_two_sum(sh, sl, z.h, z.l);
  return z;
}

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  float ch = __fmul_rn(x.h, y.h);
  float cl1 = __fmaf_rn(x.h, y.h, -ch);
  float tl = __fmul_rn(x.h, y.l);
  float cl2 = __fmaf_rn(x.l, y.h, tl);
  float cl3 = __fadd_rn(cl1, cl2);
  dfl z;
  fast_two_sum(ch, cl3, z.h, z.l);
  return z;
}

// Split a double into hi + lo floats (hi = RN(x), lo = RN(x - hi)).  Runs on
// the FP64 unit; used only outside the iteration (set-up and finish).
__device__ __forceinline__ dfl df_from_double(double x) {
  dfl r;
  r.h = __double2float_rn(x);
  r.l = __double2float_rn(x - (double)r.h);
  return r;
}
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.h + (double)a.l; }

// Compensated accumulator: running float sum s plus float compensation c.
struct cacc {
  float s, c;
};
__device__ __forceinline__ void cacc_add(cacc &A, float p, float e) {
  float s, t;
  two_sum(A.s, p, s, t);
  A.s = s;
  A.c = __fadd_rn(A.c, __fadd_rn(t, e));
}
// A += a*b for double-float a, b: exact leading product plus cross terms.
__device__ __forceinline__ void cacc_add_prod(cacc &A, dfl a, dfl b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  cacc_add(A, p, e);
}
// A += a*b for floats (the product is exact as p + e).
__device__ __forceinline__ void cacc_add_prodf(cacc &A, float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  cacc_add(A, p, e);
}
// Renormalise to a double-float.  s is the rounded running sum and c the
// accumulated rounding errors, so |c| <= |s| except when the sum cancels to
// below the accumulation's own error bound (about n^2 2^-48 of the sum of
// |terms|); FastTwoSum is exact in the first case and in the second adds
// an error of the order of ulp(c), inside that same bound.
__device__ __forceinline__ dfl cacc_get(cacc A) {
  dfl z;
  fast_two_sum(A.s, A.c, z.h, z.l);
  return z;
}

// ------------------------------------------------------------------ PF64
struct PF64 {
  using st = double;   // element in HBM
  using val = double;  // element in registers / shared memory
  using coef = double; // metric-table entry
  using scal = double; // alpha, beta
  struct sacc {
    double v;
  };
  struct dacc {
    double v;
  };
  static constexpr int kVec = 2; // elements per 16-byte vector
  static __device__ __forceinline__ val ld(const st *p) { return *p; }
  static __device__ __forceinline__ void stv(st *p, val v) { *p = v; }
  static __device__ __forceinline__ val zero() { return 0.0; }
  static __device__ __forceinline__ scal scal_from(double x) { return x; }
  static __device__ __forceinline__ val fma(scal a, val x, val y) { return ::fma(a, x, y); }
  static __device__ __forceinline__ sacc s_init(val c) { return {c}; }
  static __device__ __forceinline__ void s_add(sacc &s, coef c, val x) { s.v = ::fma(c, x, s.v); }
  static __device__ __forceinline__ val s_get(const sacc &s) { return s.v; }
  static __device__ __forceinline__ dacc d_init() { return {0.0}; }
  static __device__ __forceinline__ void d_add(dacc &d, val a, val b) { d.v = ::fma(a, b, d.v); }
  static __device__ __forceinline__ void d_addw(dacc &d, coef w, const dacc &row) {
    d.v = ::fma(w, row.v, d.v);
  }
  static __device__ __forceinline__ double d_get(const dacc &d) { return d.v; }
  static __device__ __forceinline__ void d_merge(dacc &d, const dacc &s) { d.v += s.v; }
  static __device__ __forceinline__ val from_double(double x) { return x; }
  static __device__ __forceinline__ double to_double(val v) { return v; }
  // scalar helpers of the phi-line ring solve
  static __device__ __forceinline__ dacc d_of(val v) { return {v}; }
  static __device__ __forceinline__ val one() { return 1.0; }
  static __device__ __forceinline__ val mul(val a, val b) { return a * b; }
  static __device__ __forceinline__ val sub(val a, val b) { return a - b; }
  static __device__ __forceinline__ val add(val a, val b) { return a + b; }
  static __device__ __forceinline__ val div(val a, val b) { return a / b; }
  static __device__ __forceinline__ val shfl_up(val v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
  static __device__ __forceinline__ val shfl_down(val v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
  }
  static __device__ __forceinline__ val shfl_idx(val v, int l) { return __shfl_sync(0xffffffffu, v, l); }
  // 16-byte vector of kVec elements
  static __device__ __forceinline__ void ldv(const st *p, val (&v)[kVec]) {
    double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
    v[0] = t.x;
    v[1] = t.y;
  }
  static __device__ __forceinline__ void stvv(st *p, const val (&v)[kVec]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
};

// ------------------------------------------------------------------- PDF
struct PDF {
  using st = float2;
  using val = dfl;
  using coef = float2;
  using scal = dfl;
  using sacc = cacc;
  using dacc = cacc;
  static constexpr int kVec = 2;
  static __device__ __forceinline__ val ld(const st *p) {
    float2 t = *p;
    return {t.x, t.y};
  }
  static __device__ __forceinline__ void stv(st *p, val v) { *p = make_float2(v.h, v.l); }
  static __device__ __forceinline__ val zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ scal scal_from(double x) { return df_from_double(x); }
  // y + a x: the product's leading part exactly (TwoProd) plus its cross
  // terms, added to y with one TwoSum and a final FastTwoSum (the product
  // is not renormalised on its own; same error order as SloppyDWPlusDW of
  // DWTimesDW, four operations fewer)
  static __device__ __forceinline__ val fma(scal a, val x, val y) {
    const float ph = __fmul_rn(a.h, x.h);
    float pl = __fmaf_rn(a.h, x.h, -ph);
    pl = __fmaf_rn(a.h, x.l, pl);
    pl = __fmaf_rn(a.l, x.h, pl);
    float sh, sl;
    two_sum(y.h, ph, sh, sl);
    sl = __fadd_rn(sl, __fadd_rn(y.l, pl));
    dfl z;
    fast_two_sum(sh, sl, z.h, z.l);
    return z;
  }
  static __device__ __forceinline__ sacc s_init(val c) { return {c.h, c.l}; }
  static __device__ __forceinline__ void s_add(sacc &s, coef c, val x) {
    cacc_add_prod(s, dfl{c.x, c.y}, x);
  }
  static __device__ __forceinline__ val s_get(const sacc &s) { return cacc_get(s); }
  static __device__ __forceinline__ dacc d_init() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void d_add(dacc &d, val a, val b) { cacc_add_prod(d, a, b); }
  static __device__ __forceinline__ void d_addw(dacc &d, coef w, const dacc &row) {
    cacc_add_prod(d, dfl{w.x, w.y}, cacc_get(row));
  }
  static __device__ __forceinline__ double d_get(const dacc &d) {
    return (double)d.s + (double)d.c;
  }
  static __device__ __forceinline__ void d_merge(dacc &d, const dacc &s) { cacc_add(d, s.s, s.c); }
  static __device__ __forceinline__ val from_double(double x) { return df_from_double(x); }
  static __device__ __forceinline__ double to_double(val v) { return df_to_double(v); }
  static __device__ __forceinline__ void ldv(const st *p, val (&v)[kVec]) {
    float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = {t.x, t.y};
    v[1] = {t.z, t.w};
  }
  static __device__ __forceinline__ void stvv(st *p, const val (&v)[kVec]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0].h, v[0].l, v[1].h, v[1].l);
  }
};

// ------------------------------------------------------------------ PF32
struct PF32 {
  using st = float;
  using val = float;
  using coef = float;
  using scal = float;
  struct sacc {
    float v;
  };
  using dacc = cacc; // dot products: exact float products, compensated sums
  static constexpr int kVec = 4;
  static __device__ __forceinline__ val ld(const st *p) { return *p; }
  static __device__ __forceinline__ void stv(st *p, val v) { *p = v; }
  static __device__ __forceinline__ val zero() { return 0.f; }
  static __device__ __forceinline__ scal scal_from(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ val fma(scal a, val x, val y) { return __fmaf_rn(a, x, y); }
  static __device__ __forceinline__ sacc s_init(val c) { return {c}; }
  static __device__ __forceinline__ void s_add(sacc &s, coef c, val x) { s.v = __fmaf_rn(c, x, s.v); }
  static __device__ __forceinline__ val s_get(const sacc &s) { return s.v; }
  static __device__ __forceinline__ dacc d_init() { return {0.f, 0.f}; }
  static __device__ __forceinline__ void d_add(dacc &d, val a, val b) { cacc_add_prodf(d, a, b); }
  static __device__ __forceinline__ void d_addw(dacc &d, coef w, const dacc &row) {
    cacc_add_prod(d, dfl{w, 0.f}, cacc_get(row));
  }
  static __device__ __forceinline__ double d_get(const dacc &d) {
    return (double)d.s + (double)d.c;
  }
  static __device__ __forceinline__ void d_merge(dacc &d, const dacc &s) { cacc_add(d, s.s, s.c); }
  static __device__ __forceinline__ val from_double(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ double to_double(val v) { return (double)v; }
  // scalar helpers of the phi-line ring solve
  static __device__ __forceinline__ dacc d_of(val v) { return {v, 0.f}; }
  static __device__ __forceinline__ val one() { return 1.f; }
  static __device__ __forceinline__ val mul(val a, val b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ val sub(val a, val b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ val add(val a, val b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ val div(val a, val b) { return __fdiv_rn(a, b); }
  static __device__ __forceinline__ val shfl_up(val v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
  static __device__ __forceinline__ val shfl_down(val v, int d) {
    return __shfl_down_sync(0xffffffffu, v, d);
  }
  static __device__ __forceinline__ val shfl_idx(val v, int l) { return __shfl_sync(0xffffffffu, v, l); }
  static __device__ __forceinline__ void ldv(const st *p, val (&v)[kVec]) {
    float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  static __device__ __forceinline__ void stvv(st *p, const val (&v)[kVec]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

} // namespace pot3d
