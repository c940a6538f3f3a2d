// Tensor-product ("sum-factorised") cell operators on shared-memory tiles.
//
// A tile holds, for each of RT independent slots (a slot is one real column of
// one cell), the values on a 3D tensor grid laid out [n3][n2][n1][RT] with the
// slot index fastest.  A 1D matrix Mat[mout][min] is applied along one axis;
// the three 1D factors of B = B1 (x) B1 (x) B1 (basis at Gauss-Legendre
// points) and the exact 1D stiffness/mass matrices reproduce the cell
// matrices of Eq. Hmn without forming them.  All extents are compile-time so
// the work-item decomposition costs no integer division.
#pragma once

#include "efe_internal.h"

namespace efe {

// ---------------------------------------------------------------------------
// Pair-of-binary32 ("double-word") arithmetic on the FP32 pipe.  A value is
// h + l with |l| <= ulp(h) / 2 once normalised.  The error-free transformations
// are Knuth's TwoSum, Dekker's Fast2Sum and the FMA form of TwoProd; the
// addition and multiplication of two pairs are the accurate algorithms of
// Joldes, Muller and Popescu (ACM TOMS 44, 2017: "AccurateDWPlusDW",
// relative error <= 3u^2, and "DWTimesDW3", <= 4u^2, u = 2^-24).  A chain of
// products accumulated by fma() keeps its low word unnormalised (the exact
// rounding error of every high-word addition is added into it) and fin()
// renormalises it with one TwoSum.  The _rn intrinsics keep the compiler from
// contracting or reassociating the transformations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ df32 operator+(df32 x, df32 y) {
  float sh, sl, th, tl, vh, vl, zh, zl;
  two_sum(x.h, y.h, sh, sl);
  two_sum(x.l, y.l, th, tl);
  fast_two_sum(sh, __fadd_rn(sl, th), vh, vl);
  fast_two_sum(vh, __fadd_rn(tl, vl), zh, zl);
  return df32(zh, zl);
}
__device__ __forceinline__ df32 operator*(df32 x, df32 y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);
  const float tl1 = __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.l));
  const float cl2 = __fmaf_rn(x.l, y.h, tl1);
  float zh, zl;
  fast_two_sum(ch, __fadd_rn(cl1, cl2), zh, zl);
  return df32(zh, zl);
}
__device__ __forceinline__ df32& operator+=(df32& a, df32 b) { return a = a + b; }
__device__ __forceinline__ df32& operator*=(df32& a, df32 b) { return a = a * b; }
__device__ __forceinline__ bool operator!=(df32 a, df32 b) { return a.h != b.h || a.l != b.l; }
// c + a b: exact product error and exact high-word rounding error go to the low word.
// a, b and c may be unnormalised results of earlier chains of m terms (|l| <= m ulp(h)):
// the products a.h b.l and a.l b.h then still carry ~m 2^-48 relative error, so values
// that only feed further chains or a multiplication skip fin() (operator* leaves its
// result normalised); values that meet operator+ do not.
using ::fma;   // keep the float and double overloads visible next to this one
__device__ __forceinline__ df32 fma(df32 a, df32 b, df32 c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  float s, err;
  two_sum(c.h, p, s, err);
  return df32(s, __fadd_rn(c.l, __fadd_rn(err, e)));
}
__device__ __forceinline__ df32 fin(df32 a) {
  float s, e;
  two_sum(a.h, a.l, s, e);
  return df32(s, e);
}
__device__ __forceinline__ float fin(float a) { return a; }
__device__ __forceinline__ double fin(double a) { return a; }

template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ const double* B1(const RefTables& t) { return t.B1; }
  static __device__ __forceinline__ const double* K1(const RefTables& t) { return t.K1; }
  static __device__ __forceinline__ const double* M1(const RefTables& t) { return t.M1; }
  static __device__ __forceinline__ const double* D1(const RefTables& t) { return t.D1; }
};
template <> struct Tab<df32> {
  static __device__ __forceinline__ const df32* B1(const RefTables& t) { return t.B1p; }
  static __device__ __forceinline__ const df32* K1(const RefTables& t) { return t.K1p; }
  static __device__ __forceinline__ const df32* M1(const RefTables& t) { return t.M1p; }
  static __device__ __forceinline__ const df32* D1(const RefTables& t) { return t.D1p; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ const float* B1(const RefTables& t) { return t.B1f; }
  static __device__ __forceinline__ const float* K1(const RefTables& t) { return t.K1f; }
  static __device__ __forceinline__ const float* M1(const RefTables& t) { return t.M1f; }
  static __device__ __forceinline__ const float* D1(const RefTables& t) { return t.D1f; }
};

// out[..o..] (=|+=) rs[r] * sum_m Mat[o * MIN + m] * in[..m..]   (TRANS: Mat[m * MOUT + o])
// Work items are (a, b, r) over the two untouched axes (extents NA, NB) and the slot.
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC, int NA, int NB, int SA_IN, int SB_IN,
          int SM_IN, int SA_OUT, int SB_OUT, int SM_OUT>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out, const T* mat, const T* rs) {
  constexpr int ITEMS = NA * NB * RT;
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int r = it % RT;
    const int ab = it / RT;
    const int a = ab % NA, b = ab / NA;
    const T* src = in + a * SA_IN + b * SB_IN + r;
    T v[MIN];
#pragma unroll
    for (int m = 0; m < MIN; ++m) v[m] = src[m * SM_IN];
    T* dst = out + a * SA_OUT + b * SB_OUT + r;
#pragma unroll
    for (int o = 0; o < MOUT; ++o) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < MIN; ++m) acc = fma(TRANS ? mat[m * MOUT + o] : mat[o * MIN + m], v[m], acc);
      // outputs that only feed later fma chains stay unnormalised (see fma)
      if (rs) acc = rs[r] * acc;
      if (ACC)
        dst[o * SM_OUT] += acc;
      else
        dst[o * SM_OUT] = acc;
    }
  }
}

// Apply a 1D operator along axis 1 (fastest), 2 or 3 of a tile with dims
// (N3, N2, N1) where the contracted axis has extent MIN -> MOUT.
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC, int N2, int N3>
__device__ __forceinline__ void along1(const T* in, T* out, const T* mat, const T* rs = nullptr) {
  contract<T, MIN, MOUT, RT, TRANS, ACC, N2, N3, MIN * RT, N2 * MIN * RT, RT, MOUT * RT, N2 * MOUT * RT, RT>(in, out,
                                                                                                          mat, rs);
}
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC, int N1, int N3>
__device__ __forceinline__ void along2(const T* in, T* out, const T* mat, const T* rs = nullptr) {
  contract<T, MIN, MOUT, RT, TRANS, ACC, N1, N3, RT, MIN * N1 * RT, N1 * RT, RT, MOUT * N1 * RT, N1 * RT>(in, out,
                                                                                                        mat, rs);
}
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC, int N1, int N2>
__device__ __forceinline__ void along3(const T* in, T* out, const T* mat, const T* rs = nullptr) {
  contract<T, MIN, MOUT, RT, TRANS, ACC, N1, N2, RT, N1 * RT, N2 * N1 * RT, RT, N1 * RT, N2 * N1 * RT>(in, out, mat,
                                                                                                     rs);
}

// Kinetic part of a box cell, 1/2 int grad N_I . grad N_J applied to X:
//   Y = ax K1(x)M1(x)M1 X + ay M1(x)K1(x)M1 X + az M1(x)M1(x)K1 X   (axis order x, y, z)
// with ax = hy hz / (4 hx) etc. given per slot.  X in A, result in B, C and D
// scratch; all P1^3 * RT.
template <typename T, int P1, int RT>
__device__ __forceinline__ void kinetic_tile(const RefTables& tab, const T* A, T* B, T* C, T* D, const T* ax,
                                             const T* ay, const T* az) {
  const T* K1 = Tab<T>::K1(tab);
  const T* M1 = Tab<T>::M1(tab);
  along3<T, P1, P1, RT, false, false, P1, P1>(A, B, M1);            // B = M_3 X
  along3<T, P1, P1, RT, false, false, P1, P1>(A, C, K1);            // C = K_3 X
  __syncthreads();
  along2<T, P1, P1, RT, false, false, P1, P1>(B, D, K1, ay);        // D = ay K_2 M_3 X
  __syncthreads();
  along2<T, P1, P1, RT, false, true, P1, P1>(C, D, M1, az);         // D += az M_2 K_3 X
  __syncthreads();
  along2<T, P1, P1, RT, false, false, P1, P1>(B, C, M1);            // C = M_2 M_3 X
  __syncthreads();
  along1<T, P1, P1, RT, false, false, P1, P1>(D, B, M1);            // B = M_1 D
  __syncthreads();
  along1<T, P1, P1, RT, false, true, P1, P1>(C, B, K1, ax);         // B += ax K_1 M_2 M_3 X
  __syncthreads();
}

// Values at the Gauss-Legendre points: A (P1^3 slots) -> C (NQ1^3), D scratch.
template <typename T, int P1, int NQ1, int RT>
__device__ __forceinline__ void interp_fwd(const RefTables& tab, const T* A, T* C, T* D) {
  const T* B1 = Tab<T>::B1(tab);
  along1<T, P1, NQ1, RT, false, false, P1, P1>(A, C, B1);           // (P1, P1, NQ1)
  __syncthreads();
  along2<T, P1, NQ1, RT, false, false, NQ1, P1>(C, D, B1);          // (P1, NQ1, NQ1)
  __syncthreads();
  along3<T, P1, NQ1, RT, false, false, NQ1, NQ1>(D, C, B1);         // (NQ1, NQ1, NQ1)
  __syncthreads();
}

// Projection back: C (NQ1^3) -> B (P1^3), added when ACC; D and E scratch
// (E may alias C).
template <typename T, int P1, int NQ1, int RT, bool ACC>
__device__ __forceinline__ void interp_bwd(const RefTables& tab, const T* C, T* B, T* D, T* E) {
  const T* B1 = Tab<T>::B1(tab);
  along3<T, NQ1, P1, RT, true, false, NQ1, NQ1>(C, D, B1);          // (P1, NQ1, NQ1)
  __syncthreads();
  along2<T, NQ1, P1, RT, true, false, NQ1, P1>(D, E, B1);           // (P1, P1, NQ1)
  __syncthreads();
  along1<T, NQ1, P1, RT, true, ACC, P1, P1>(E, B, B1);              // (P1, P1, P1)
  __syncthreads();
}

// Classical cell operator of one tile, kinetic plus v-weighted mass:
//   Y = cx K_1 M_2 M_3 X + cy M_1 K_2 M_3 X + cz M_1 M_2 K_3 X + B^T diag(W) B X
// (subscript = axis; cx = hy hz / (4 hx) etc.), ordered so that every output
// is one accumulation chain and no stage adds into a stored tile:
//   G  = (B1^T (x) B1^T) [W (B1 (x) B1 (x) B1) X]          axes 3, 2 of the back projection
//   A <- cx M_3 X,  B <- cy M_3 X,  D <- cz K_3 X           (one pass over axis-3 lines)
//   B <- K_2 B + M_2 D,  A <- M_2 A                         (one pass over axis-2 lines)
//   D <- K_1 A + M_1 B + B1^T_1 G                           (one pass over axis-1 lines)
// X in A (overwritten), result in D; B, C scratch; W the cell's weights [NQ1^3].
template <typename T, int P1, int NQ1, int RT>
__device__ __forceinline__ void cell_operator_tile(const RefTables& tab, T* A, T* B, T* C, T* D,
                                                   const T* __restrict__ W, T cx, T cy, T cz) {
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  const T* B1 = Tab<T>::B1(tab);
  const T* K1 = Tab<T>::K1(tab);
  const T* M1 = Tab<T>::M1(tab);
  interp_fwd<T, P1, NQ1, RT>(tab, A, C, D);
  for (int it = threadIdx.x; it < S3 * RT; it += blockDim.x) C[it] *= W[it / RT];
  __syncthreads();
  along3<T, NQ1, P1, RT, true, false, NQ1, NQ1>(C, D, B1);          // (P1, NQ1, NQ1)
  __syncthreads();
  along2<T, NQ1, P1, RT, true, false, NQ1, P1>(D, C, B1);           // G: (P1, P1, NQ1)
  __syncthreads();
  constexpr int ITEMS = P1 * P1 * RT;
  // axis-3 lines: offset (i2 P1 + i1) RT + r, stride P1^2 RT
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    constexpr int S = P1 * P1 * RT;
    T v[P1];
#pragma unroll
    for (int m = 0; m < P1; ++m) v[m] = A[it + m * S];
#pragma unroll
    for (int o = 0; o < P1; ++o) {
      T p = T(0), q = T(0);
#pragma unroll
      for (int m = 0; m < P1; ++m) {
        p = fma(M1[o * P1 + m], v[m], p);
        q = fma(K1[o * P1 + m], v[m], q);
      }
      A[it + o * S] = cx * p;
      B[it + o * S] = cy * p;
      D[it + o * S] = cz * q;
    }
  }
  __syncthreads();
  // axis-2 lines: offset (i3 P1^2 + i1) RT + r, stride P1 RT
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    constexpr int S = P1 * RT;
    const int r = it % RT, i1 = (it / RT) % P1, i3 = it / (RT * P1);
    const int off = (i3 * P1 * P1 + i1) * RT + r;
    T a[P1], b[P1], d[P1];
#pragma unroll
    for (int m = 0; m < P1; ++m) {
      a[m] = A[off + m * S];
      b[m] = B[off + m * S];
      d[m] = D[off + m * S];
    }
#pragma unroll
    for (int o = 0; o < P1; ++o) {
      T y = T(0), e = T(0);
#pragma unroll
      for (int m = 0; m < P1; ++m) {
        y = fma(K1[o * P1 + m], b[m], y);
        e = fma(M1[o * P1 + m], a[m], e);
      }
#pragma unroll
      for (int m = 0; m < P1; ++m) y = fma(M1[o * P1 + m], d[m], y);
      B[off + o * S] = y;
      A[off + o * S] = e;
    }
  }
  __syncthreads();
  // axis-1 lines: offset (i3 P1 + i2) P1 RT + r (G: (i3 P1 + i2) NQ1 RT + r), stride RT
  for (int it = threadIdx.x; it < ITEMS; it += blockDim.x) {
    const int r = it % RT, l23 = it / RT;
    const int off = l23 * P1 * RT + r;
    const int offg = l23 * NQ1 * RT + r;
    T a[P1], b[P1], g[NQ1];
#pragma unroll
    for (int m = 0; m < P1; ++m) {
      a[m] = A[off + m * RT];
      b[m] = B[off + m * RT];
    }
#pragma unroll
    for (int q = 0; q < NQ1; ++q) g[q] = C[offg + q * RT];
#pragma unroll
    for (int o = 0; o < P1; ++o) {
      T y = T(0);
#pragma unroll
      for (int m = 0; m < P1; ++m) {
        y = fma(K1[o * P1 + m], a[m], y);
        y = fma(M1[o * P1 + m], b[m], y);
      }
#pragma unroll
      for (int q = 0; q < NQ1; ++q) y = fma(B1[q * P1 + o], g[q], y);
      D[off + o * RT] = fin(y);
    }
  }
  __syncthreads();
}

// IEEE-754 conversions between binary64 and binary32 on the integer pipes
// (the FP64 unit of this GPU issues two operations per clock per SM, so the
// hardware conversions would bind the float32 kernels).  Both follow the bit
// layouts of the formats: f64_to_f32_rn rounds to nearest even, flushes
// results below the smallest normal float to signed zero and saturates to
// infinity; f32_to_f64 is exact for normal floats and maps subnormal floats to
// signed zero.
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu) - 896;          // binary32 biased exponent
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 mantissa bits
  const unsigned rest = lo & 0x1FFFFFFFu;                   // 29 dropped bits
  unsigned r = ((unsigned)e << 23) + m;
  r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  r = e <= 0 ? 0u : r;
  r = (e >= 255 || r >= 0x7F800000u) ? 0x7F800000u : r;
  return __uint_as_float(sign | r);
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned m = u & 0x7FFFFFu;
  unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
  unsigned lo = m << 29;
  if (e == 0u) { hi = sign; lo = 0u; }
  if (e == 255u) hi = sign | 0x7FF00000u | (m >> 3);
  return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return f64_to_f32_rn(x); }
template <typename T> __device__ __forceinline__ double to_f64(T x);
template <> __device__ __forceinline__ double to_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ double to_f64<float>(float x) { return f32_to_f64(x); }
// x = h + l with h the nearest binary32 and l the nearest binary32 to x - h (one float64 subtraction)
template <> __device__ __forceinline__ df32 from_f64<df32>(double x) {
  const float h = f64_to_f32_rn(x);
  return df32(h, f64_to_f32_rn(x - f32_to_f64(h)));
}
template <> __device__ __forceinline__ double to_f64<df32>(df32 x) { return f32_to_f64(x.h) + f32_to_f64(x.l); }

// x = h + l on the integer pipes, without rounding: h holds the leading 24 significant bits of x,
// l the next 24 (truncated), so |x - (h + l)| < 2^-47 |x| for |x| > 1e-23; parts below the binary32
// normal range are flushed to zero (absolute error < 1e-37), magnitudes beyond it become infinite.  One float64 value costs ~15 integer operations and no FP64-pipe work.
__device__ __forceinline__ df32 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);                 // biased binary64 exponent
  const unsigned mh = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // next 23 bits after the leading one
  const unsigned rest = lo & 0x1FFFFFFFu;                    // the 29 bits below them
  const int eh = e - 896;                                    // binary32 biased exponent of h
  const float h = eh <= 0 ? 0.0f : __uint_as_float(sign | (eh < 255 ? ((unsigned)eh << 23) | mh : 0x7F800000u));
  float l = 0.0f;
  if (rest != 0u) {
    const int pm = 31 - __clz((int)rest);                    // position of the leading one of rest
    const unsigned m = pm <= 23 ? rest << (23 - pm) : rest >> (pm - 23);
    const int el = pm + e - 948;                             // rest * 2^(e - 1075) in binary32
    if (el > 0 && el < 255) l = __uint_as_float(sign | ((unsigned)el << 23) | (m & 0x7FFFFFu));
  }
  return df32(h, l);
}

// Gathered operands: FP64 products enter the fma chains through the exact split for pairs.
template <typename T> __device__ __forceinline__ T from_f64_split(double x);
template <> __device__ __forceinline__ double from_f64_split<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64_split<float>(double x) { return f64_to_f32_rn(x); }
template <> __device__ __forceinline__ df32 from_f64_split<df32>(double x) { return split_f64(x); }

}  // namespace efe
