// The classical cell operator and the enrichment coupling on the fifth-generation
// tensor cores (precision EFE_TC).
//
// The apply of Hbar (Eq. TDKSDiscrete2, H = P^T H_ext P written out block by block
// as in k_apply.cu) needs, per cell c,
//   y^C_c = H_c x^C_c + E_c x^E_c,      y^E_c = E_c^T x^C_c,
// with H_c the dense cell matrix (kinetic stiffness + v-weighted mass, Eqs. Hmn and
// VeffDiscrete; P1^3 <= 128 nodes at degree <= 4) and E_c the cell's block of the
// classical-enriched coupling.  These are dense contractions, so they run on the
// tensor cores with an exact-product splitting: every float64 operand is scaled by a
// power of two per row (rows of [H_c E_c], rows of E_c^T) or per column (of
// [x^C; x^E]), rounded to 31 bits and cut into four bf16 slices of 7 + 8 + 8 + 8
// bits.  A product of two slices is exact in binary32.  Slice pairs whose indices
// sum to 0 are accumulated in one tensor-memory accumulator and pairs summing to 1
// in a second: both sums are exact (at most 2 x 176 terms on a grid of 2^-14 resp.
// 2^-22, below 2^24 grid steps).  Pairs summing to 2, 3 or 4 go to a third
// accumulator, whose binary32 rounding is ~2^-39 of the scales; pairs summing to 5
// or 6 are dropped (each below 2^-38 of the scales).  The result is
// 2^(row + column exponent) (acc0 + acc1 + acc2), formed in float64.  Per element of
// y the error is a few 2^-31 of sum_k |A_ik| max_k |x_k|.  Two choices matter here:
// a pair (k, l) carries up to 2^(2 - 8(k + l)) of the scales whatever the size of
// its product, and a typical entry is ~2^-7 of its row's largest, so stopping at
// k + l = 3 would leave binary32-level (2^-30 of the scales) errors; and with one
// accumulator for every pair past the first, the exact but large cross terms
// a0 b1 + a1 b0 would round the finer groups away at binary32's relative 2^-24.
//
// Layout: the A operands (H_c slices, E_c and E_c^T slices) are written when the
// operator is built, directly in the shared-memory image the MMA reads (no-swizzle
// K-major core matrices, see tc.cuh), so the apply copies them with plain 16-byte
// copies.  The apply is a persistent kernel, one CTA of 512 threads per SM:
//   gather x_bar^C and x^E, x^C = D x_bar^C, per-column exponents, split into 4 slices
//   (smem); all float64 work is done on the integer pipes from bit patterns (GB300's
//   float64 pipe is ~1/64 of its float32 pipe).  The output-side D is folded into the
//   rows of H_c and E_c when they are built.
//   for slice i of H_c / E_c / E_c^T (copied into smem, next slices prefetched to L2):
//       one thread issues the MMAs of the pairs (i, j), i + j <= 4, commits to an
//       mbarrier; all threads wait (bounded)
//   epilogue: accumulators -> exact 64-bit fixed point -> float64 -> y_bar^C, y^E
//   (atomic adds)
#include <cstdio>
#include <vector>

#include "efe_internal.h"
#include "tc.cuh"

namespace efe {

namespace {

constexpr int kSlices = 4;
constexpr int kMaxGroup = 4;                    // slice pairs (i, j) with i + j <= 4 are formed
constexpr int kK = 128;                         // padded node dimension
constexpr int kSliceBytes = 128 * kK * 2;       // one 128 x 128 bf16 slice
constexpr int kMaxKE = 48;                      // enrichment functions per cell
constexpr int kMaxN = 96;                       // real columns per batch member
constexpr int kZero = -100000;                  // exponent of an all-zero row or column
constexpr uint32_t kWaitLimit = 1u << 22;       // mbarrier polls before giving up (seconds)

// shared-memory map of the apply kernel (bytes)
constexpr int kXs = 0;                                   // 4 slices x 128 x 128 (x^C, K-major)
constexpr int kXEs = kXs + kSlices * kSliceBytes;        // 4 slices x 96 x 48   (x^E, K-major)
constexpr int kXEslice = kMaxN * kMaxKE * 2;
constexpr int kAH = kXEs + kSlices * kXEslice;           // H_c slice i
constexpr int kAEA = kAH + kSliceBytes;                  // E_c slice i      (128 x KEp)
constexpr int kAET = kAEA + 128 * kMaxKE * 2;            // E_c^T slice i    (KEp x 128)
constexpr int kMisc = kAET + kMaxKE * kK * 2;
constexpr int kApplySmem = kMisc + 128 * 8 * 2 + 128 * 4 + (96 + 96 + 128 + 48 + 48) * 4 + 16;
constexpr int kApplyThreads = 512;
constexpr int kMaxPer = 26;                     // nodes gathered per thread (even; 512 / 96 >= 5 groups)

__device__ __forceinline__ long long q31(double v, int e) { return e == kZero ? 0LL : tc::q31_bits(v, e); }
__device__ __forceinline__ int exp_of_max(double mx) {
  const int be = tc::biased_exp(mx);
  return (be == 0 || be - 1022 < -990) ? kZero : tc::scale_exp(be);
}
// eight consecutive values of one core-matrix row, scaled by 2^-e, stored as four
// 16-byte slice rows at dst + s * stride
__device__ __forceinline__ void store_slices8(const double* v, int e, unsigned char* dst, long long stride) {
  uint32_t w[kSlices][4];
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    uint16_t a[kSlices], b[kSlices];
    tc::split4(q31(v[t], e), a);
    tc::split4(q31(v[t + 1], e), b);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) w[s][t / 2] = (uint32_t)a[s] | ((uint32_t)b[s] << 16);
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s)
    *reinterpret_cast<uint4*>(dst + s * stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

}  // namespace

// ----------------------------------------------------------------------------
// build: dense H_c in float64 by sum factorisation, row exponents, slices of H_c,
// E_c (rows scaled with H_c's) and E_c^T (rows scaled per function).
//   M_c[i][j] = sum_q W_q prod_d B1[q_d][i_d] B1[q_d][j_d]
//   K_c[i][j] = kx K1 M1 M1 + ky M1 K1 M1 + kz M1 M1 K1        (axis order x, y, z)
// One block of 256 threads per (cell, member).
// ----------------------------------------------------------------------------
template <int P1, int NQ1>
__global__ void __launch_bounds__(256)
k_tc_build(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ W64, double kin,
           const int* __restrict__ pair_start, const double* __restrict__ E64, long long n_pairs,
           const double* __restrict__ Dsc, const long long* __restrict__ eoff, long long e_total,
           unsigned char* __restrict__ tcH,
           int* __restrict__ tcRexp, unsigned char* __restrict__ tcE, int* __restrict__ tcHexp) {
  constexpr int NN = P1 * P1 * P1;
  constexpr int S3 = NQ1 * NQ1 * NQ1;
  constexpr int PP = P1 * P1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Ws = reinterpret_cast<double*>(smem_raw);
  double* P = Ws + S3;                 // [a a'][q]
  double* T1 = P + PP * NQ1;           // [a a'][q2 + NQ1 q3]
  double* T2 = T1 + PP * NQ1 * NQ1;    // [(a a') PP + (b b')][q3]
  double* H = T2 + PP * PP * NQ1;      // [NN][NN]
  double* Dn = H + NN * NN;           // D = mask / sqrt(M) at the cell's nodes
  int* rexp = reinterpret_cast<int*>(Dn + 128);
  int* hexp = rexp + 128;
  const int c = blockIdx.x, m = blockIdx.y, tid = threadIdx.x;
  int cx, cy, cz;
  cell_ijk(mesh, c, cx, cy, cz);
  const double hx = mesh.h[cx], hy = mesh.h[mesh.ncx + cy], hz = mesh.h[mesh.ncx + mesh.ncy + cz];
  const double kx = kin * hy * hz / (4.0 * hx), ky = kin * hx * hz / (4.0 * hy), kz = kin * hx * hy / (4.0 * hz);
  for (int q = tid; q < S3; q += blockDim.x) Ws[q] = W64[((long long)m * mesh.nc + c) * S3 + q];
  for (int l = tid; l < NN; l += blockDim.x) Dn[l] = Dsc[node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / PP)];
  for (int it = tid; it < PP * NQ1; it += blockDim.x) {
    const int q = it % NQ1, aa = it / NQ1;
    P[it] = tab.B1[q * P1 + aa / P1] * tab.B1[q * P1 + aa % P1];
  }
  __syncthreads();
  for (int it = tid; it < PP * NQ1 * NQ1; it += blockDim.x) {
    const int r = it % (NQ1 * NQ1), aa = it / (NQ1 * NQ1);
    double acc = 0.0;
    for (int q1 = 0; q1 < NQ1; ++q1) acc += P[aa * NQ1 + q1] * Ws[q1 + NQ1 * r];
    T1[it] = acc;
  }
  __syncthreads();
  for (int it = tid; it < PP * PP * NQ1; it += blockDim.x) {
    const int q3 = it % NQ1, t = it / NQ1, bb = t % PP, aa = t / PP;
    double acc = 0.0;
    for (int q2 = 0; q2 < NQ1; ++q2) acc += P[bb * NQ1 + q2] * T1[aa * NQ1 * NQ1 + q2 + NQ1 * q3];
    T2[it] = acc;
  }
  __syncthreads();
  for (int it = tid; it < NN * NN; it += blockDim.x) {
    const int i = it / NN, j = it % NN;
    const int a = i % P1, b = (i / P1) % P1, cc = i / PP;
    const int a2 = j % P1, b2 = (j / P1) % P1, c2 = j / PP;
    const int aa = a * P1 + a2, bb = b * P1 + b2, ccp = cc * P1 + c2;
    double acc = 0.0;
    for (int q3 = 0; q3 < NQ1; ++q3) acc += P[ccp * NQ1 + q3] * T2[(aa * PP + bb) * NQ1 + q3];
    const double Ka = tab.K1[a * P1 + a2], Kb = tab.K1[b * P1 + b2], Kc = tab.K1[cc * P1 + c2];
    const double Ma = tab.M1[a * P1 + a2], Mb = tab.M1[b * P1 + b2], Mc = tab.M1[cc * P1 + c2];
    acc += kx * Ka * Mb * Mc + ky * Ma * Kb * Mc + kz * Ma * Mb * Kc;
    H[it] = Dn[i] * acc;   // the output side of the Loewdin scaling, folded in (rows keep one scale)
  }
  int p0 = 0, np = 0;
  if (pair_start) {
    p0 = pair_start[c];
    np = pair_start[c + 1] - p0;
  }
  const double* Ec = E64 + ((long long)m * n_pairs + p0) * NN;
  __syncthreads();
  // row exponents, joint over the row of H_c and the row of E_c (one accumulator)
  for (int i = tid; i < 128; i += blockDim.x) {
    double mx = 0.0;
    if (i < NN) {
      for (int j = 0; j < NN; ++j) mx = fmax(mx, fabs(H[i * NN + j]));
      for (int f = 0; f < np; ++f) mx = fmax(mx, fabs(Dn[i] * Ec[(long long)f * NN + i]));
    }
    rexp[i] = i < NN ? exp_of_max(mx) : kZero;
    tcRexp[((long long)m * mesh.nc + c) * 128 + i] = rexp[i];
  }
  for (int f = tid; f < np; f += blockDim.x) {
    double mx = 0.0;
    for (int i = 0; i < NN; ++i) mx = fmax(mx, fabs(Ec[(long long)f * NN + i]));
    hexp[f] = exp_of_max(mx);
    tcHexp[(long long)m * n_pairs + p0 + f] = hexp[f];
  }
  __syncthreads();
  // H_c slices: item = one 16-byte core-matrix row (i, 8 consecutive k), consecutive
  // items at consecutive addresses
  unsigned char* Hc = tcH + ((long long)m * mesh.nc + c) * kSlices * kSliceBytes;
  for (int it = tid; it < 128 * (kK / 8); it += blockDim.x) {
    const int i8 = it & 7, kc = (it >> 3) & 15, ig = it >> 7;
    const int i = ig * 8 + i8;
    double v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int k = kc * 8 + t;
      v[t] = (i < NN && k < NN) ? H[i * NN + k] : 0.0;
    }
    store_slices8(v, rexp[i], Hc + tc::kmajor_offset(i, kc * 8, 2048), kSliceBytes);
  }
  if (np > 0) {
    const int KEp = (np + 15) & ~15;
    const long long eb = 256LL * KEp;   // bytes of one 128 x KEp slice
    unsigned char* Eb = tcE + ((long long)m * e_total + eoff[c]) * 2048;
    // E_c (rows i, K = f), rows scaled with H_c's
    const int nfc = KEp / 8;
    for (int it = tid; it < 128 * nfc; it += blockDim.x) {
      const int i8 = it & 7, fc = (it >> 3) % nfc, ig = (it >> 3) / nfc;
      const int i = ig * 8 + i8;
      double v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int f = fc * 8 + t;
        v[t] = (i < NN && f < np) ? Dn[i] * Ec[(long long)f * NN + i] : 0.0;
      }
      store_slices8(v, rexp[i], Eb + tc::kmajor_offset(i, fc * 8, 16 * KEp), eb);
    }
    // E_c^T (rows f, K = i), rows scaled by hexp
    for (int it = tid; it < KEp * (kK / 8); it += blockDim.x) {
      const int f8 = it & 7, ic = (it >> 3) & 15, fg = it >> 7;
      const int f = fg * 8 + f8;
      double v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = ic * 8 + t;
        v[t] = (f < np && i < NN) ? Ec[(long long)f * NN + i] : 0.0;
      }
      store_slices8(v, f < np ? hexp[f] : kZero, Eb + 4 * eb + tc::kmajor_offset(f, ic * 8, 2048), eb);
    }
  }
}

// ----------------------------------------------------------------------------
// apply (persistent; one CTA per SM)
// ----------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(kApplyThreads, 1)
k_tc_apply(const MeshView mesh, const double* __restrict__ X, double* __restrict__ Y, long long ld2, int cols, int nm,
           int batch, const double* __restrict__ Dsc, const unsigned char* __restrict__ tcH,
           const int* __restrict__ tcRexp, const unsigned char* __restrict__ tcE, long long e_total,
           const long long* __restrict__ eoff, const int* __restrict__ tcHexp, const int* __restrict__ pair_start,
           const int* __restrict__ pair_fn, long long n_pairs, const double* __restrict__ xE, double* __restrict__ yE,
           int* __restrict__ err, const int* __restrict__ gate) {
  constexpr int NN = P1 * P1 * P1;
  constexpr int NT = kApplyThreads;
  extern __shared__ __align__(1024) unsigned char sm[];
  long long* gS = reinterpret_cast<long long*>(sm + kMisc);   // [128] global node of each cell node
  unsigned long long* dm = reinterpret_cast<unsigned long long*>(gS + 128);   // [128] significand of D
  int* de = reinterpret_cast<int*>(dm + 128);                 // [128] exponent of D
  int* colmax = de + 128;                                     // [96]
  int* fexp = colmax + 96;                                    // [96] column exponents
  int* rexp = fexp + 96;                                      // [128] row exponents
  int* hexp = rexp + 128;                                     // [48] E_c^T row exponents
  int* fns = hexp + 48;                                       // [48] enrichment functions of the cell
  uint64_t* mbar = reinterpret_cast<uint64_t*>(fns + 48);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tbase + 1);
  if (gate && *gate == 0) return;   // every Lanczos column has converged (graph-captured loops)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // gather mapping: thread (group g, column n) owns column n of the nodes
  // [g per, (g + 1) per); per is even so that node pairs share a 4-byte slot
  const int G = NT / cols;
  const int per = 2 * ((NN + 2 * G - 1) / (2 * G));
  const int gg = tid / cols, gn = tid - gg * cols;
  const bool active = gg < G;
  // operand images start zeroed: rows n >= cols and nodes l >= NN of x^C stay zero
  for (int o = tid * 16; o < kAH; o += NT * 16) *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    *abort_flag = 0;
  }
  if (warp == 0) tc::tmem_alloc(tbase, 512);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tbase;
  uint32_t phase = 0;
  const uint32_t idm = tc::idesc_bf16(128, nm);
  const long long nwork = (long long)mesh.nc * batch;
  const uint32_t xs = tc::smem_u32(sm + kXs), xes = tc::smem_u32(sm + kXEs), ah = tc::smem_u32(sm + kAH),
                 aea = tc::smem_u32(sm + kAEA), aet = tc::smem_u32(sm + kAET);
  bool aborted = false;
  for (long long w = blockIdx.x; w < nwork && !aborted; w += gridDim.x) {
    const int c = (int)(w % mesh.nc), m = (int)(w / mesh.nc);
    const int col0 = m * cols;
    int p0 = 0, np = 0;
    if (pair_start) {
      p0 = pair_start[c];
      np = pair_start[c + 1] - p0;
    }
    const int KEp = (np + 15) & ~15;
    const long long eb = 256LL * KEp;
    const unsigned char* Hc = tcH + ((long long)m * mesh.nc + c) * kSlices * kSliceBytes;
    const unsigned char* Ec = np > 0 ? tcE + ((long long)m * e_total + eoff[c]) * 2048 : nullptr;
    auto load_set = [&](int i) {
      for (int o = tid * 16; o < kSliceBytes; o += NT * 16) tc::cp_async16(sm + kAH + o, Hc + i * kSliceBytes + o);
      if (np > 0)
        for (int o = tid * 16; o < eb; o += NT * 16) {
          tc::cp_async16(sm + kAEA + o, Ec + i * eb + o);
          tc::cp_async16(sm + kAET + o, Ec + 4 * eb + i * eb + o);
        }
    };
    load_set(0);
    // the remaining slices of this cell and the first of the next one, into L2
    for (int o = tid * 128; o < 3 * kSliceBytes; o += NT * 128)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(Hc + kSliceBytes + o));
    if (np > 0)
      for (int o = tid * 128; o < 3 * eb; o += NT * 128) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Ec + eb + o));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Ec + 5 * eb + o));
      }
    if (w + gridDim.x < nwork) {
      const unsigned char* Hn = tcH + (w + gridDim.x) * kSlices * kSliceBytes;
      for (int o = tid * 128; o < kSliceBytes; o += NT * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(Hn + o));
    }
    int cx, cy, cz;
    cell_ijk(mesh, c, cx, cy, cz);
    for (int l = tid; l < 128; l += NT) {
      if (l < NN) {
        const long long g = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1));
        gS[l] = g;
        const tc::Wide d = tc::wide_of(Dsc[g]);
        dm[l] = d.m;
        de[l] = d.e;
      }
      rexp[l] = tcRexp[((long long)m * mesh.nc + c) * 128 + l];
    }
    for (int f = tid; f < np; f += NT) {
      fns[f] = pair_fn[p0 + f];
      hexp[f] = tcHexp[(long long)m * n_pairs + p0 + f];
    }
    for (int n = tid; n < 96; n += NT) colmax[n] = 0;
    if (np > 0)
      for (int o = tid * 16; o < kSlices * kXEslice; o += NT * 16)
        *reinterpret_cast<uint4*>(sm + kXEs + o) = make_uint4(0, 0, 0, 0);
    __syncthreads();
    // gather x_bar^C into registers, every load issued first; x^C = D x_bar^C is formed
    // (64-bit significand product) on the integer pipes
    const int l0 = gg * per;
    double xv[kMaxPer];
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j) {
      xv[j] = 0.0;
      if (active && j < per && l0 + j < NN) xv[j] = X[gS[l0 + j] * ld2 + col0 + gn];
    }
    int kmax = 0;
#pragma unroll
    for (int j = 0; j < kMaxPer; ++j)
      if (active && j < per && l0 + j < NN)
        kmax = max(kmax, tc::wide_key(tc::wide_mul(tc::wide_of(xv[j]), dm[l0 + j], de[l0 + j])));
    for (int f = gg; active && f < np; f += G)
      kmax = max(kmax, tc::wide_key(tc::wide_of(xE[(long long)fns[f] * ld2 + col0 + gn])));
    if (active) atomicMax(&colmax[gn], kmax);
    __syncthreads();
    for (int n = tid; n < 96; n += NT) {
      const int k = colmax[n];   // floor(log2 max|x|) + 2048
      fexp[n] = k == 0 ? kZero : k - 2048 + 1;
    }
    __syncthreads();
    // slices of x^C (rows n, K = node), two nodes per 4-byte store, and of x^E
    if (active) {
      const int fe = fexp[gn];
#pragma unroll
      for (int j = 0; j < kMaxPer; j += 2) {
        const int l = l0 + j;
        if (j < per && l < NN) {
          uint16_t s0[kSlices], s1[kSlices];
          const tc::Wide x0 = tc::wide_mul(tc::wide_of(xv[j]), dm[l], de[l]);
          tc::split4(fe == kZero ? 0LL : tc::q31_wide(x0, fe), s0);
          if (l + 1 < NN) {
            const tc::Wide x1 = tc::wide_mul(tc::wide_of(xv[j + 1]), dm[l + 1], de[l + 1]);
            tc::split4(fe == kZero ? 0LL : tc::q31_wide(x1, fe), s1);
          } else {
#pragma unroll
            for (int k = 0; k < kSlices; ++k) s1[k] = 0;
          }
          const uint32_t off = tc::kmajor_offset(gn, l, 2048);
#pragma unroll
          for (int k = 0; k < kSlices; ++k)
            *reinterpret_cast<uint32_t*>(sm + kXs + k * kSliceBytes + off) = (uint32_t)s0[k] | ((uint32_t)s1[k] << 16);
        }
      }
      for (int f = gg; f < np; f += G) {
        uint16_t s[kSlices];
        tc::split4(fe == kZero ? 0LL : tc::q31_wide(tc::wide_of(xE[(long long)fns[f] * ld2 + col0 + gn]), fe), s);
        const uint32_t off = tc::kmajor_offset(gn, f, 16 * KEp);
#pragma unroll
        for (int k = 0; k < kSlices; ++k) *reinterpret_cast<uint16_t*>(sm + kXEs + k * kXEslice + off) = s[k];
      }
    }
    // the next cell's rows of x_bar, into L2
    if (w + gridDim.x < nwork) {
      const long long w2 = w + gridDim.x;
      const int c2 = (int)(w2 % mesh.nc), m2 = (int)(w2 / mesh.nc);
      int ex, ey, ez;
      cell_ijk(mesh, c2, ex, ey, ez);
      const int lines = (cols * 8 + 127) / 128 + 1;   // 128-byte steps plus the row's last entry
      for (int it = tid; it < NN * lines; it += NT) {
        const int l = it / lines, q = it - l * lines;
        const long long g = node_index(mesh, ex, ey, ez, l % P1, (l / P1) % P1, l / (P1 * P1));
        const char* row = reinterpret_cast<const char*>(X + g * ld2 + (long long)m2 * cols);
        const int off = q + 1 < lines ? 128 * q : cols * 8 - 8;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
      }
    }
    tc::cp_async_wait_all();
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    for (int i = 0; i < kSlices; ++i) {
      if (tid == 0) {
        tc::fence_after_sync();
        for (int j = 0; j < kSlices && i + j <= kMaxGroup; ++j) {
          const int gsum = i + j;
          const uint32_t acc = gsum == 0 ? 0u : gsum == 1 ? 96u : 192u;
          const uint32_t dacc = tm + acc;
          const uint32_t dT = tm + 288u + acc / 2;
          const bool first = i == 0 && j <= 2;   // first pair of each accumulator's group
          for (int ks = 0; ks < kK / 16; ++ks)
            tc::mma_bf16(dacc, tc::smem_desc(ah + 256 * ks, tc::kLBO, 2048),
                         tc::smem_desc(xs + j * kSliceBytes + 256 * ks, tc::kLBO, 2048), idm, !(first && ks == 0));
          if (np > 0) {
            const uint32_t sbo = 16 * KEp;
            for (int ks = 0; ks < KEp / 16; ++ks)
              tc::mma_bf16(dacc, tc::smem_desc(aea + 256 * ks, tc::kLBO, sbo),
                           tc::smem_desc(xes + j * kXEslice + 256 * ks, tc::kLBO, sbo), idm, true);
            const uint32_t idt = tc::idesc_bf16(128, KEp);
            for (int ks = 0; ks < kK / 16; ++ks)
              tc::mma_bf16(dT, tc::smem_desc(xs + j * kSliceBytes + 256 * ks, tc::kLBO, 2048),
                           tc::smem_desc(aet + 256 * ks, tc::kLBO, 2048), idt, !(first && ks == 0));
          }
        }
        tc::mma_commit(mbar);
      }
      const bool ok = tc::mbar_wait(mbar, phase, kWaitLimit);
      phase ^= 1u;
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 1);
      }
      tc::fence_after_sync();
      if (i + 1 < kSlices) {
        load_set(i + 1);
        tc::cp_async_wait_all();
        tc::fence_proxy_async();
      }
      tc::fence_before_sync();
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
    }
    if (aborted) break;
    tc::fence_after_sync();
    // epilogue: warp w reads lanes 32 (w % 4) ..; the four warps of a lane group take
    // 8-column chunks in turn
    const int lg = warp & 3, qw = warp >> 2;
    const int r = 32 * lg + lane;
    const uint32_t lane_addr = (uint32_t)(32 * lg) << 16;
    const long long gr = r < NN ? gS[r] : 0;
    const int re = rexp[r];
    for (int ch = qw; ch * 8 < nm; ch += 4) {
      const int col = 8 * ch;
      float a0[8], a1[8], a2[8];
      tc::tmem_ld8(tm + lane_addr + col, a0);
      tc::tmem_ld8(tm + lane_addr + 96 + col, a1);
      tc::tmem_ld8(tm + lane_addr + 192 + col, a2);
      if (r < NN && re != kZero) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int n = col + t;
          if (n >= cols) break;
          const int fe = fexp[n];
          if (fe == kZero) continue;
          // acc0 and acc1 are exact on the 2^-46 grid, acc2 to its last bit above it
          const long long I = tc::fixed_of_float(a0[t], 46) + tc::fixed_of_float(a1[t], 46) +
                              tc::fixed_of_float(a2[t], 46);
          if (I != 0) atomicAdd(&Y[gr * ld2 + col0 + n], tc::double_of_fixed(I, re + fe - 46));
        }
      }
    }
    if (np > 0) {
      const int n = r;
      const int fe = n < cols ? fexp[n] : kZero;
      for (int ch = qw; ch * 8 < KEp; ch += 4) {
        float t0[8], t1[8], t2[8];
        tc::tmem_ld8(tm + lane_addr + 288 + 8 * ch, t0);
        tc::tmem_ld8(tm + lane_addr + 336 + 8 * ch, t1);
        tc::tmem_ld8(tm + lane_addr + 384 + 8 * ch, t2);
        if (fe != kZero) {
#pragma unroll
          for (int t = 0; t < 8; ++t) {
            const int f = 8 * ch + t;
            if (f >= np) break;
            if (hexp[f] == kZero) continue;
            const long long I = tc::fixed_of_float(t0[t], 46) + tc::fixed_of_float(t1[t], 46) +
                                tc::fixed_of_float(t2[t], 46);
            if (I != 0) atomicAdd(&yE[(long long)fns[f] * ld2 + col0 + n], tc::double_of_fixed(I, fe + hexp[f] - 46));
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (aborted && tid == 0) tc::mbar_wait(mbar, phase, kWaitLimit);   // MMAs still in flight
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tm, 512);
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
template <typename F>
static cudaError_t set_smem_tc(F f, size_t bytes) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

const char* tc_unsupported(const Ctx& c, int cols_member) {
  if (c.p > 4) return "EFE_TC needs degree <= 4 (at most 128 nodes per cell)";
  if (c.max_pairs_per_cell > kMaxKE) return "EFE_TC needs at most 48 enrichment functions per cell";
  if (cols_member > kMaxN) return "EFE_TC needs at most 96 real columns (48 orbitals) per batch member";
  return nullptr;
}

static cudaError_t tc_alloc(Ctx& c, int batch) {
  TcState& t = c.tc;
  if (t.eoff == nullptr) {
    std::vector<int> ps(c.nc + 1, 0);
    if (c.n_pairs > 0)
      EFE_CUDA_TRY(cudaMemcpy(ps.data(), c.d_pair_start, sizeof(int) * (c.nc + 1), cudaMemcpyDeviceToHost));
    std::vector<long long> eo(c.nc + 1, 0);
    for (int i = 0; i < c.nc; ++i) eo[i + 1] = eo[i] + (((ps[i + 1] - ps[i]) + 15) & ~15);
    t.e_total = eo[c.nc];
    EFE_CUDA_TRY(cudaMalloc(&t.eoff, sizeof(long long) * (c.nc + 1)));
    EFE_CUDA_TRY(cudaMemcpy(t.eoff, eo.data(), sizeof(long long) * (c.nc + 1), cudaMemcpyHostToDevice));
    EFE_CUDA_TRY(cudaMalloc(&t.err, sizeof(int)));
    EFE_CUDA_TRY(cudaMemset(t.err, 0, sizeof(int)));
  }
  if (t.batch != batch) {
    cudaFree(t.H); cudaFree(t.rexp); cudaFree(t.E); cudaFree(t.hexp);
    t.H = nullptr; t.rexp = nullptr; t.E = nullptr; t.hexp = nullptr;
    t.batch = 0;
    EFE_CUDA_TRY(cudaMalloc(&t.H, (size_t)batch * c.nc * kSlices * kSliceBytes));
    EFE_CUDA_TRY(cudaMalloc(&t.rexp, sizeof(int) * (size_t)batch * c.nc * 128));
    EFE_CUDA_TRY(cudaMalloc(&t.E, (size_t)batch * (t.e_total > 0 ? t.e_total : 1) * 2048));
    EFE_CUDA_TRY(cudaMalloc(&t.hexp, sizeof(int) * (size_t)batch * (c.n_pairs > 0 ? c.n_pairs : 1)));
    t.batch = batch;
    c.ws_gen++;   // captured graphs hold the old pointers
  }
  return cudaSuccess;
}

template <int P1, int NQ1>
static cudaError_t tc_build_impl(Ctx& c, int batch, cudaStream_t s) {
  EFE_CUDA_TRY(tc_alloc(c, batch));
  constexpr int NN = P1 * P1 * P1, S3 = NQ1 * NQ1 * NQ1, PP = P1 * P1;
  const size_t sm = sizeof(double) * (S3 + PP * NQ1 + PP * NQ1 * NQ1 + PP * PP * NQ1 + NN * NN + 128) + sizeof(int) * (128 + 48);
  auto f = k_tc_build<P1, NQ1>;
  EFE_CUDA_TRY(set_smem_tc(f, sm));
  dim3 grid(c.nc, batch);
  f<<<grid, 256, sm, s>>>(c.tab, c.mesh, c.op.W64, c.op.kin, c.n_pairs > 0 ? c.d_pair_start : nullptr, c.op.E64,
                          c.n_pairs, c.d_Dsc, c.tc.eoff, c.tc.e_total, c.tc.H, c.tc.rexp, c.tc.E, c.tc.hexp);
  note_launch();
  return cudaGetLastError();
}

template <int P1>
static cudaError_t tc_apply_impl(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, cudaStream_t s) {
  const long long ld2 = 2 * ld;
  const int batch = c.op.batch;
  const int cols = (int)(2 * n_cols / batch);
  const int ncols2 = (int)(2 * n_cols);
  EFE_CUDA_TRY(cudaMemset2DAsync(Y, sizeof(double) * ld2, 0, sizeof(double) * ncols2, c.n_dof, s));
  if (c.nE > 0) {
    EFE_CUDA_TRY(cudaMemsetAsync(c.d_yE, 0, sizeof(double) * c.nE * ld2, s));
    EFE_CUDA_TRY(launch_enr_pre(c, X, ld2, ncols2, s));
  }
  if (c.tc.n_sm == 0) EFE_CUDA_TRY(cudaDeviceGetAttribute(&c.tc.n_sm, cudaDevAttrMultiProcessorCount, c.device));
  const long long nwork = (long long)c.nc * batch;
  const unsigned grid = (unsigned)(nwork < c.tc.n_sm ? nwork : c.tc.n_sm);
  auto f = k_tc_apply<P1>;
  EFE_CUDA_TRY(set_smem_tc(f, kApplySmem));
  const int nm = (cols + 15) & ~15;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!c.apply_gate) prof_pair(c, e0, e1);
  if (e0) EFE_CUDA_TRY(cudaEventRecord(e0, s));
  f<<<grid, kApplyThreads, kApplySmem, s>>>(c.mesh, X, Y, ld2, cols, nm, batch, c.d_Dsc, c.tc.H, c.tc.rexp, c.tc.E, c.tc.e_total,
                                  c.tc.eoff, c.tc.hexp, c.n_pairs > 0 ? c.d_pair_start : nullptr, c.d_pair_fn,
                                  c.n_pairs, c.d_xE, c.d_yE, c.tc.err, c.apply_gate);
  note_launch();
  EFE_CUDA_TRY(cudaGetLastError());
  if (e1) EFE_CUDA_TRY(cudaEventRecord(e1, s));
  if (c.nE > 0) EFE_CUDA_TRY(launch_enr_post(c, Y, ld2, ncols2, cols, s));
  return cudaSuccess;
}

cudaError_t launch_tc_build(Ctx& c, int batch, cudaStream_t s) {
  switch (c.p) {
    case 2: return tc_build_impl<3, 4>(c, batch, s);
    case 3: return tc_build_impl<4, 5>(c, batch, s);
    case 4: return tc_build_impl<5, 6>(c, batch, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tc_apply(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, cudaStream_t s) {
  switch (c.p) {
    case 2: return tc_apply_impl<3>(c, X, Y, n_cols, ld, s);
    case 3: return tc_apply_impl<4>(c, X, Y, n_cols, ld, s);
    case 4: return tc_apply_impl<5>(c, X, Y, n_cols, ld, s);
    default: return cudaErrorInvalidValue;
  }
}

void tc_free(TcState& t) {
  cudaFree(t.H); cudaFree(t.rexp); cudaFree(t.E); cudaFree(t.hexp); cudaFree(t.eoff); cudaFree(t.err);
  t = TcState{};
}

}  // namespace efe
