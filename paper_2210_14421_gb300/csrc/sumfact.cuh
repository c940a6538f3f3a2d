// Tensor-product ("sum-factorised") cell operators on shared-memory tiles.
//
// A tile holds, for each of RT independent slots (a slot is one real column of
// one cell), the values on a 3D tensor grid laid out [n3][n2][n1][RT] with the
// slot index fastest.  A 1D matrix Mat[mout][min] is applied along one axis;
// the three 1D factors of B = B1 (x) B1 (x) B1 (basis at Gauss-Legendre
// points), of the derivative tables and of the exact 1D stiffness/mass
// matrices reproduce the cell matrices of Eq. Hmn without forming them.
#pragma once

#include "efe_internal.h"

namespace efe {

template <typename T> struct Tab;
template <> struct Tab<double> {
  static __device__ __forceinline__ const double* B1(const RefTables& t) { return t.B1; }
  static __device__ __forceinline__ const double* K1(const RefTables& t) { return t.K1; }
  static __device__ __forceinline__ const double* M1(const RefTables& t) { return t.M1; }
  static __device__ __forceinline__ const double* D1(const RefTables& t) { return t.D1; }
};
template <> struct Tab<float> {
  static __device__ __forceinline__ const float* B1(const RefTables& t) { return t.B1f; }
  static __device__ __forceinline__ const float* K1(const RefTables& t) { return t.K1f; }
  static __device__ __forceinline__ const float* M1(const RefTables& t) { return t.M1f; }
  static __device__ __forceinline__ const float* D1(const RefTables& t) { return t.D1f; }
};

// out[..o..] (=|+=) rs[r] * sum_m Mat[o * MIN + m] * in[..m..]   (TRANS: Mat[m * MOUT + o])
// Work items are (a, b, r) over the two untouched axes and the slot.
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out, const T* mat, int nA,
                                         int nB, int sA_in, int sB_in, int sM_in, int sA_out, int sB_out,
                                         int sM_out, const T* rs) {
  const int items = nA * nB * RT;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int r = it % RT;
    const int ab = it / RT;
    const int a = ab % nA, b = ab / nA;
    const T* src = in + a * sA_in + b * sB_in + r;
    T v[MIN];
#pragma unroll
    for (int m = 0; m < MIN; ++m) v[m] = src[m * sM_in];
    const T scale = rs ? rs[r] : T(1);
    T* dst = out + a * sA_out + b * sB_out + r;
#pragma unroll
    for (int o = 0; o < MOUT; ++o) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < MIN; ++m) acc = fma(TRANS ? mat[m * MOUT + o] : mat[o * MIN + m], v[m], acc);
      if (ACC)
        dst[o * sM_out] += scale * acc;
      else
        dst[o * sM_out] = scale * acc;
    }
  }
}

// Apply a 1D operator along axis 1 (fastest), 2 or 3 of a tile with dims
// (N3, N2, N1) where the contracted axis has extent MIN -> MOUT.
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC>
__device__ __forceinline__ void along1(const T* in, T* out, const T* mat, int N2, int N3, const T* rs = nullptr) {
  contract<T, MIN, MOUT, RT, TRANS, ACC>(in, out, mat, N2, N3, MIN * RT, N2 * MIN * RT, RT, MOUT * RT,
                                         N2 * MOUT * RT, RT, rs);
}
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC>
__device__ __forceinline__ void along2(const T* in, T* out, const T* mat, int N1, int N3, const T* rs = nullptr) {
  contract<T, MIN, MOUT, RT, TRANS, ACC>(in, out, mat, N1, N3, RT, MIN * N1 * RT, N1 * RT, RT, MOUT * N1 * RT,
                                         N1 * RT, rs);
}
template <typename T, int MIN, int MOUT, int RT, bool TRANS, bool ACC>
__device__ __forceinline__ void along3(const T* in, T* out, const T* mat, int N1, int N2, const T* rs = nullptr) {
  contract<T, MIN, MOUT, RT, TRANS, ACC>(in, out, mat, N1, N2, RT, N1 * RT, N2 * N1 * RT, RT, N1 * RT,
                                         N2 * N1 * RT, rs);
}

// Kinetic part of a box cell, 1/2 int grad N_I . grad N_J applied to X:
//   Y = ax K1(x)M1(x)M1 X + ay M1(x)K1(x)M1 X + az M1(x)M1(x)K1 X   (axis order x, y, z)
// with ax = hy hz / (4 hx) etc. given per slot.  Buffers: X in A, result in B,
// C and D scratch; all P1^3 * RT.  ACC_OUT adds into B instead of overwriting.
template <typename T, int P1, int RT>
__device__ __forceinline__ void kinetic_tile(const RefTables& tab, const T* A, T* B, T* C, T* D, const T* ax,
                                             const T* ay, const T* az) {
  const T* K1 = Tab<T>::K1(tab);
  const T* M1 = Tab<T>::M1(tab);
  along3<T, P1, P1, RT, false, false>(A, B, M1, P1, P1);            // B = M_3 X
  along3<T, P1, P1, RT, false, false>(A, C, K1, P1, P1);            // C = K_3 X
  __syncthreads();
  along2<T, P1, P1, RT, false, false>(B, D, K1, P1, P1, ay);        // D = ay K_2 M_3 X
  __syncthreads();
  along2<T, P1, P1, RT, false, true>(C, D, M1, P1, P1, az);         // D += az M_2 K_3 X
  __syncthreads();
  along2<T, P1, P1, RT, false, false>(B, C, M1, P1, P1);            // C = M_2 M_3 X
  __syncthreads();
  along1<T, P1, P1, RT, false, false>(D, B, M1, P1, P1);            // B = M_1 D
  __syncthreads();
  along1<T, P1, P1, RT, false, true>(C, B, K1, P1, P1, ax);         // B += ax K_1 M_2 M_3 X
  __syncthreads();
}

// Values at the Gauss-Legendre points: U = B X (A -> C via D), then optional
// pointwise weights, then B^T back and accumulated into B.
template <typename T, int P1, int NQ1, int RT>
__device__ __forceinline__ void interp_fwd(const RefTables& tab, const T* A, T* C, T* D) {
  const T* B1 = Tab<T>::B1(tab);
  along1<T, P1, NQ1, RT, false, false>(A, C, B1, P1, P1);           // (P1, P1, NQ1)
  __syncthreads();
  along2<T, P1, NQ1, RT, false, false>(C, D, B1, NQ1, P1);          // (P1, NQ1, NQ1)
  __syncthreads();
  along3<T, P1, NQ1, RT, false, false>(D, C, B1, NQ1, NQ1);         // (NQ1, NQ1, NQ1)
  __syncthreads();
}

template <typename T, int P1, int NQ1, int RT, bool ACC>
__device__ __forceinline__ void interp_bwd(const RefTables& tab, const T* C, T* B, T* D, T* E) {
  const T* B1 = Tab<T>::B1(tab);
  along3<T, NQ1, P1, RT, true, false>(C, D, B1, NQ1, NQ1);          // (P1, NQ1, NQ1)
  __syncthreads();
  along2<T, NQ1, P1, RT, true, false>(D, E, B1, NQ1, P1);           // (P1, P1, NQ1)
  __syncthreads();
  along1<T, NQ1, P1, RT, true, ACC>(E, B, B1, P1, P1);              // (P1, P1, P1)
  __syncthreads();
}

}  // namespace efe
