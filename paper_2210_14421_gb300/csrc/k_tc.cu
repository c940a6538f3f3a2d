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
// power of two per row (rows of H_c, rows of E_c, rows of E_c^T) or per column (of
// x^C, of x^E; each its own), rounded to 31 bits and cut into four bf16 slices on
// the grids 2^-7, 2^-15, 2^-23, 2^-31.  A product of two slices is exact in
// binary32.  Slice pairs whose indices sum to 0 are accumulated in one
// tensor-memory accumulator and pairs summing to 1 in a second: both sums are exact
// (at most 2 x 128 terms on a grid of 2^-14 resp. 2^-22, below 2^24 grid steps).
// Pairs summing to 2, 3 or 4 go to a third accumulator, whose binary32 rounding is
// ~2^-39 of the scales; pairs summing to 5 or 6 are dropped (each below 2^-38 of the
// scales).  A product is 2^(row + column exponent) (acc0 + acc1 + acc2); the three
// binary32 partial sums are added as an unevaluated float pair (error-free TwoSum
// chains) and the pair is turned into one float64 on the integer pipes.  Per element
// of y the error is a few 2^-31 of sum_k |A_ik| max_k |x_k| for each product apart.
//
// Separate scales: in cells near a nucleus the enrichment part of an orbital is many
// orders of magnitude larger than its classical part, so x^C and x^E have their own
// column exponents (and E_c its own row exponents).  The products therefore have
// their own accumulators: first the E pass (E_c x^E and E_c^T x^C), whose classical
// part is parked in tensor memory as a float pair, then the H pass (H_c x^C); the two
// float pairs are brought to the larger of the two exponents and summed before the
// one float64 value per output is formed.
//
// Layout: the A operands (H_c slices, E_c and E_c^T slices) are written when the
// operator is built, directly in the shared-memory image the MMA reads (no-swizzle
// K-major core matrices, see tc.cuh), with the Loewdin scaling D = mask / sqrt(M)
// folded into both sides of H_c and into E_c, so the apply reads x_bar as stored.
// The A images stream into a two-slot ring with bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier).  Cells with more than 48
// enrichment functions are split into work items of at most 48 functions (the first
// one carries H_c), and an apply over more than 96 columns runs in column blocks.
// The apply is persistent, one CTA per SM, warp-specialised:
//   24 work warps: gather x_bar^C (rows of the cell's nodes; the next cell's rows are
//     prefetched into L2) and x^E, per-column exponents, digit extraction into 4
//     bf16 slices (shared memory); after the MMAs the epilogues: accumulators ->
//     float pair -> float64, E_c^T x^C to y^E (atomic adds), y_c staged in shared
//     memory and scattered row by row (coalesced atomic adds; plain stores for the
//     interior nodes of a cell that is its own only work item);
//   1 issuer warp: streams the A slices (E pass: E_c slice i with E_c^T slice i;
//     H pass: H_c slice i) and issues, from one lane, the MMAs of the slice pairs
//     (i, j), i + j <= 4, committing to mbarriers that free ring slots and release
//     the epilogues.  Every wait is bounded: a wait that gives up sets an error flag
//     the host reads (EFE_ERR_TIMEOUT), waits (bounded) for the copies and MMAs in
//     flight and frees the tensor memory before returning.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "efe_internal.h"
#include "sumfact.cuh"
#include "tc.cuh"

namespace efe {

namespace {

constexpr int kSlices = 4;
constexpr int kMaxGroup = 4;                    // slice pairs (i, j) with i + j <= 4 are formed
constexpr int kK = 128;                         // padded node dimension
constexpr int kSliceBytes = 128 * kK * 2;       // one 128 x 128 bf16 slice of H_c
constexpr int kMaxKE = 48;                      // enrichment functions per cell
constexpr int kMaxN = 96;                       // real columns per batch member
constexpr int kZero = -100000;                  // exponent of an all-zero row or column
constexpr uint32_t kWaitLimit = 1u << 22;       // mbarrier polls before giving up (seconds)

// the apply kernel: kWork / 32 work warps (a multiple of 4: the tensor-memory lane quarters) and one
// issuer warp (on the Na8-like workload, per apply: 12 + 1 warps 9.9 ms, 16 + 1 8.5 ms, 24 + 1 7.9 ms;
// 24 work warps run at 72 registers per thread)
#ifndef EFE_TC_WORK_WARPS
#define EFE_TC_WORK_WARPS 24
#endif
constexpr int kWork = 32 * EFE_TC_WORK_WARPS;
constexpr int kApplyThreads = kWork + 32;
constexpr int kWPQ = EFE_TC_WORK_WARPS / 4;                 // work warps per lane quarter
constexpr int kNQ = (kMaxN / 8 + kWPQ - 1) / kWPQ;          // 8-column chunks per thread in an epilogue
constexpr int kNK = ((kK / 8) * kMaxN + kWork - 1) / kWork; // gather items per thread
constexpr int kNSlot = 2;                                   // ring slots for the streamed A operands
// shared-memory map of the apply kernel (bytes)
constexpr int kXslice = kMaxN * kK * 2;                     // x^C slice: 96 rows (columns n) x 128 nodes
constexpr int kXs = 0;                                      // 4 x^C slices; y_c staging after the MMAs
constexpr int kXEslice = kMaxN * kMaxKE * 2;                // x^E slice: 96 rows x 48 functions
constexpr int kXEs = kXs + kSlices * kXslice;
constexpr int kRing = kXEs + kSlices * kXEslice;            // kNSlot x 32 KB
constexpr int kMisc = kRing + kNSlot * kSliceBytes;
constexpr int kStageLd = kMaxN + 1;                         // staging row stride (doubles; odd: no bank conflicts)
static_assert(125 * kStageLd * 8 <= kSlices * kXslice, "y_c staging (at most 125 nodes) must fit the x^C slices");
// misc block: the metadata of the cell being processed and of the next one (two buffers)
constexpr int kMgS = kMisc;                                 // long long [2][128] offset of each node's row in X, Y
constexpr int kMrH = kMgS + 2 * 128 * 8;                    // int [2][128] H_c row exponents
constexpr int kMrE = kMrH + 2 * 128 * 4;                    // int [2][128] E_c row exponents
constexpr int kMhx = kMrE + 2 * 128 * 4;                    // int [2][48] E_c^T row exponents
constexpr int kMfn = kMhx + 2 * kMaxKE * 4;                 // int [2][48] enrichment functions of the cell
constexpr int kMcC = kMfn + 2 * kMaxKE * 4;                 // int [96] column maxima of |x^C| (binary32 bits)
constexpr int kMcE = kMcC + kMaxN * 4;                      // int [96] column maxima of |x^E|
constexpr int kMfC = kMcE + kMaxN * 4;                      // int [96] column exponents of x^C
constexpr int kMfE = kMfC + kMaxN * 4;                      // int [96] column exponents of x^E
constexpr int kMbar = kMfE + kMaxN * 4;                     // uint64 [10] mbarriers
constexpr int kMtm = kMbar + 10 * 8;                        // uint32 tensor-memory base, int abort flag
constexpr int kApplySmem = kMtm + 16;
static_assert(kApplySmem <= 232448, "apply kernel exceeds the shared memory of a CTA");
// mbarrier indices
enum { kBFull0 = 0, kBEmpty0 = kNSlot, kBXready = 2 * kNSlot, kBAccE, kBDrainedE, kBAccH, kBFin };
static_assert(kBFin < 10, "mbarrier block too small");

// Work items of the apply: a cell with more than kMaxKE enrichment functions is processed as
// several items of at most kMaxKE functions each; the first item of a cell also carries H_c.
struct TcItems {
  int n;                   // items per batch member
  const int* cell;         // [n] the item's cell
  const int* p0;           // [n] its first cell-function pair (global pair index)
  const int* np;           // [n] its pairs
  const int* flags;        // [n] bit 0: carries H_c; bit 1: the only item of its cell
  const long long* eoff;   // [n + 1] offsets of the items' enrichment data (units of 2048 bytes)
  const int* first;        // [nc + 1] first item of each cell
};
constexpr int kItemH = 1, kItemSolo = 2;

__device__ __forceinline__ long long q31(double v, int e) { return e == kZero ? 0LL : tc::q31_bits(v, e); }
__device__ __forceinline__ int exp_of_max(double mx) {
  const int be = tc::biased_exp(mx);
  return (be == 0 || be - 1022 < -990) ? kZero : tc::scale_exp(be);
}
// column exponent from the binary32 bits of a column's largest |value|: |x| < 2^e
__device__ __forceinline__ int exp_of_maxbits(int bits) {
  if (bits <= 0) return kZero;
  const int e = (bits >> 23) - 126;
  return e < -125 ? kZero : (e > 126 ? 126 : e);
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
// eight consecutive values (a_t + b_t) 2^-e of one core-matrix row as four 16-byte slice rows
__device__ __forceinline__ void store_digits8(const float* a, const float* b, float sc, unsigned char* dst,
                                              int stride) {
  uint32_t w[kSlices][4];
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    uint32_t d0[kSlices], d1[kSlices];
    tc::digits4(__fmul_rn(a[t], sc), __fmul_rn(b[t], sc), d0);
    tc::digits4(__fmul_rn(a[t + 1], sc), __fmul_rn(b[t + 1], sc), d1);
#pragma unroll
    for (int s = 0; s < kSlices; ++s) w[s][t / 2] = tc::pack_hi16(d0[s], d1[s]);
  }
#pragma unroll
  for (int s = 0; s < kSlices; ++s)
    *reinterpret_cast<uint4*>(dst + s * stride) = make_uint4(w[s][0], w[s][1], w[s][2], w[s][3]);
}

}  // namespace

// ----------------------------------------------------------------------------
// build: dense H_c in float64 by sum factorisation, row exponents, slices of H_c,
// E_c (rows scaled by their own exponents) and E_c^T (rows scaled per function).
//   M_c[i][j] = sum_q W_q prod_d B1[q_d][i_d] B1[q_d][j_d]
//   K_c[i][j] = kx K1 M1 M1 + ky M1 K1 M1 + kz M1 M1 K1        (axis order x, y, z)
// One block of 256 threads per (cell, member).  The enrichment data of a cell are laid
// out slice by slice, [E_c slice i | E_c^T slice i] for i = 0..3, so that each stage of
// the apply's E pass is one contiguous copy.
// ----------------------------------------------------------------------------
template <int P1, int NQ1>
__global__ void __launch_bounds__(256)
k_tc_build(const __grid_constant__ RefTables tab, const MeshView mesh, const double* __restrict__ W64, double kin,
           const int* __restrict__ pair_start, const double* __restrict__ E64, long long n_pairs,
           const double* __restrict__ Dsc, const TcItems items, long long e_total,
           unsigned char* __restrict__ tcH, int* __restrict__ tcRexpH, int* __restrict__ tcRexpE,
           unsigned char* __restrict__ tcE, int* __restrict__ tcHexp) {
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
  int* rexpH = reinterpret_cast<int*>(Dn + 128);
  int* rexpE = rexpH + 128;
  int* hexp = rexpE + 128;
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
    H[it] = Dn[i] * acc * Dn[j];   // both sides of the Loewdin scaling folded in: the apply gathers x_bar
  }
  int p0c = 0, npc = 0;
  if (pair_start) {
    p0c = pair_start[c];
    npc = pair_start[c + 1] - p0c;
  }
  __syncthreads();
  // H_c row exponents
  for (int i = tid; i < 128; i += blockDim.x) {
    double mh = 0.0;
    if (i < NN)
      for (int j = 0; j < NN; ++j) mh = fmax(mh, fabs(H[i * NN + j]));
    rexpH[i] = i < NN ? exp_of_max(mh) : kZero;
    tcRexpH[((long long)m * mesh.nc + c) * 128 + i] = rexpH[i];
  }
  // E_c^T row exponents (per cell-function pair)
  for (int f = tid; f < npc; f += blockDim.x) {
    const double* Ef = E64 + ((long long)m * n_pairs + p0c + f) * NN;
    double mx = 0.0;
    for (int i = 0; i < NN; ++i) mx = fmax(mx, fabs(Ef[i] * Dn[i]));
    tcHexp[(long long)m * n_pairs + p0c + f] = exp_of_max(mx);
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
    store_slices8(v, rexpH[i], Hc + tc::kmajor_offset(i, kc * 8, 2048), kSliceBytes);
  }
  // the enrichment data of each of the cell's work items
  if (npc > 0) {
    for (int k = items.first[c]; k < items.first[c + 1]; ++k) {
      const int p0 = items.p0[k], np = items.np[k];
      const double* Ec = E64 + ((long long)m * n_pairs + p0) * NN;
      const int* hx = tcHexp + (long long)m * n_pairs + p0;
      __syncthreads();
      for (int i = tid; i < 128; i += blockDim.x) {   // E_c rows of this item: their own exponents
        double me = 0.0;
        if (i < NN)
          for (int f = 0; f < np; ++f) me = fmax(me, fabs(Dn[i] * Ec[(long long)f * NN + i]));
        rexpE[i] = i < NN ? exp_of_max(me) : kZero;
        tcRexpE[((long long)m * items.n + k) * 128 + i] = rexpE[i];
      }
      for (int f = tid; f < np; f += blockDim.x) hexp[f] = hx[f];
      __syncthreads();
      const int KEp = (np + 15) & ~15;
      const long long eb = 256LL * KEp;   // bytes of one 128 x KEp slice
      unsigned char* Eb = tcE + ((long long)m * e_total + items.eoff[k]) * 2048;
      // E_c (rows i, K = f), rows scaled by rexpE; slice s at Eb + 2 s eb
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
        store_slices8(v, rexpE[i], Eb + tc::kmajor_offset(i, fc * 8, 16 * KEp), 2 * eb);
      }
      // E_c^T D (rows f, K = i; the input side of the Loewdin scaling folded in), rows scaled by
      // hexp; slice s at Eb + (2 s + 1) eb
      for (int it = tid; it < KEp * (kK / 8); it += blockDim.x) {
        const int f8 = it & 7, ic = (it >> 3) & 15, fg = it >> 7;
        const int f = fg * 8 + f8;
        double v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int i = ic * 8 + t;
          v[t] = (f < np && i < NN) ? Ec[(long long)f * NN + i] * Dn[i] : 0.0;
        }
        store_slices8(v, f < np ? hexp[f] : kZero, Eb + eb + tc::kmajor_offset(f, ic * 8, 2048), 2 * eb);
      }
    }
  }
}

// x_bar of one cell into registers: item it = tid + k kWork is (chunk it / cols of 8 nodes, column
// it % cols); gS: offsets of the cell's node rows (column offset of the member included)
template <int NN>
__device__ __forceinline__ void gather_rows(const double* __restrict__ X, const long long* gS, int tid, int cols,
                                            int nitem, double (&v)[kNK][8]) {
#pragma unroll
  for (int k = 0; k < kNK; ++k) {
    const int it = tid + k * kWork;
    const int ch = it / cols, n = it - (it / cols) * cols;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int l = ch * 8 + t;
      v[k][t] = (it < nitem && l < NN) ? X[gS[l] + n] : 0.0;
    }
  }
}

// ----------------------------------------------------------------------------
// apply (persistent; one CTA per SM; 24 work warps + 1 issuer warp)
// ----------------------------------------------------------------------------
template <int P1>
__global__ void __launch_bounds__(kApplyThreads, 1)
k_tc_apply(const MeshView mesh, const double* __restrict__ X, double* __restrict__ Y, long long ld2, int cols, int nm,
           int batch, const double* __restrict__ Dsc, const unsigned char* __restrict__ tcH,
           const int* __restrict__ tcRexpH, const int* __restrict__ tcRexpE, const unsigned char* __restrict__ tcE,
           long long e_total, const TcItems items, const int* __restrict__ tcHexp,
           const int* __restrict__ pair_fn, long long n_pairs,
           const double* __restrict__ xE, double* __restrict__ yE, int* __restrict__ err,
           const int* __restrict__ gate, uint32_t wlim) {
  constexpr int NN = P1 * P1 * P1;
  extern __shared__ __align__(1024) unsigned char sm[];
  long long* gS2 = reinterpret_cast<long long*>(sm + kMgS);
  int* rexpH2 = reinterpret_cast<int*>(sm + kMrH);
  int* rexpE2 = reinterpret_cast<int*>(sm + kMrE);
  int* hexp2 = reinterpret_cast<int*>(sm + kMhx);
  int* fns2 = reinterpret_cast<int*>(sm + kMfn);
  int* cmaxC = reinterpret_cast<int*>(sm + kMcC);
  int* cmaxE = reinterpret_cast<int*>(sm + kMcE);
  int* fC = reinterpret_cast<int*>(sm + kMfC);
  int* fE = reinterpret_cast<int*>(sm + kMfE);
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kMbar);
  uint32_t* tbase = reinterpret_cast<uint32_t*>(sm + kMtm);
  // abort flag: written only before, and read only after, a barrier of the work warps (so that they
  // all leave the cell loop at the same barrier); the issuer warp only reads it
  volatile int* wabort = reinterpret_cast<volatile int*>(sm + kMtm + 4);
  double* stage = reinterpret_cast<double*>(sm + kXs);
  if (gate && *gate == 0) return;   // every Lanczos column has converged (graph-captured loops)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // operand images start zeroed: padding rows and nodes l >= NN stay finite
  for (int o = tid * 16; o < kRing; o += kApplyThreads * 16) *reinterpret_cast<uint4*>(sm + o) = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    for (int b = 0; b < kNSlot; ++b) {
      tc::mbar_init(&bar[kBFull0 + b], 1);
      tc::mbar_init(&bar[kBEmpty0 + b], 1);
    }
    tc::mbar_init(&bar[kBXready], 1);
    tc::mbar_init(&bar[kBAccE], 1);
    tc::mbar_init(&bar[kBDrainedE], 1);
    tc::mbar_init(&bar[kBAccH], 1);
    tc::mbar_init(&bar[kBFin], 1);
    *wabort = 0;
  }
  if (warp == 0) tc::tmem_alloc(tbase, 512);
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tm = *tbase;
  const long long nwork = (long long)items.n * batch;   // (item, member) pairs
  const uint32_t xs = tc::smem_u32(sm + kXs), xes = tc::smem_u32(sm + kXEs), ring = tc::smem_u32(sm + kRing);

  if (warp == kWork / 32) {
    // ------------------------------------------------------------ issuer warp
    // The whole warp runs the loops (operands stay warp-uniform); lane 0 waits on the mbarriers and
    // its result is broadcast, lane 0 issues the copies, MMAs and commits.
    // progress waits give up after wlim polls; the final waits for work in flight after kWaitLimit
    auto wait_n = [&](uint64_t* b, uint32_t par, uint32_t limit) {
      bool ok = true;
      if (lane == 0) ok = tc::mbar_wait(b, par, limit);
      return __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
    };
    auto wait = [&](uint64_t* b, uint32_t par) { return wait_n(b, par, wlim); };
    auto item_np = [&](long long w) { return items.np[(int)(w % items.n)]; };
    auto item_h = [&](long long w) { return (items.flags[(int)(w % items.n)] & kItemH) != 0; };
    auto n_stages = [&](long long w) { return (item_np(w) > 0 ? kSlices : 0) + (item_h(w) ? kSlices : 0); };
    // stage s of an item: E pass stages 0..3 (items coupled to enrichment functions), then the H
    // pass stages (items that carry H_c); the ring is refilled NSLOT - 1 stages ahead of the MMAs
    long long cw = blockIdx.x;   // copy cursor: item and stage
    int cst = 0, cnp = cw < nwork ? item_np(cw) : 0, cns = cw < nwork ? n_stages(cw) : 0;
    long long issued = 0, consumed = 0;
    uint32_t fparb = 0, eparb = 0;   // phase parities of the full / empty barriers, bit = slot
    uint32_t xpar = 0, dpar = 0;
    auto issue_copy = [&]() -> bool {
      if (cw >= nwork) return true;
      const int slot = (int)(issued % kNSlot);
      if (issued >= kNSlot) {
        if (!wait(&bar[kBEmpty0 + slot], (eparb >> slot) & 1u)) return false;
        eparb ^= 1u << slot;
      }
      const int it = (int)(cw % items.n), m = (int)(cw / items.n);
      const int c = items.cell[it];
      const unsigned char* src;
      uint32_t bytes;
      if (cnp > 0 && cst < kSlices) {
        const long long eb = 256LL * ((cnp + 15) & ~15);
        src = tcE + ((long long)m * e_total + items.eoff[it]) * 2048 + 2 * cst * eb;
        bytes = (uint32_t)(2 * eb);
      } else {
        const int i = cnp > 0 ? cst - kSlices : cst;
        src = tcH + ((long long)m * mesh.nc + c) * kSlices * kSliceBytes + (long long)i * kSliceBytes;
        bytes = kSliceBytes;
      }
      if (lane == 0) {
        tc::mbar_expect_tx(&bar[kBFull0 + slot], bytes);
        tc::bulk_g2s(sm + kRing + slot * kSliceBytes, src, bytes, &bar[kBFull0 + slot]);
      }
      ++issued;
      if (++cst == cns) {
        cst = 0;
        cw += gridDim.x;
        cnp = cw < nwork ? item_np(cw) : 0;
        cns = cw < nwork ? n_stages(cw) : 0;
      }
      return true;
    };
    bool ok = true;
    for (int k = 0; k < kNSlot - 1 && ok; ++k) ok = issue_copy();
    const uint32_t idH = tc::idesc_bf16(128, nm);
    // x^C slice j as the B operand of H_c x^C and the A operand of E_c^T x^C: descriptor dX0 + j dXs
    const uint64_t dX0 = tc::smem_desc(xs, tc::kLBO, 2048);
    constexpr uint64_t dXs = (uint64_t)(kXslice >> 4);
    for (long long w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
      const int np = item_np(w);
      const bool hasH = item_h(w);
      const int KEp = (np + 15) & ~15;
      const uint32_t eb = 256u * (uint32_t)KEp;
      // the next item's operator data, into L2
      if (w + gridDim.x < nwork && lane == 0) {
        const long long w2 = w + gridDim.x;
        const int it2 = (int)(w2 % items.n), m2 = (int)(w2 / items.n);
        if (item_h(w2))
          tc::bulk_prefetch_l2(tcH + ((long long)m2 * mesh.nc + items.cell[it2]) * kSlices * kSliceBytes,
                               kSlices * kSliceBytes);
        const int np2 = item_np(w2);
        if (np2 > 0)
          tc::bulk_prefetch_l2(tcE + ((long long)m2 * e_total + items.eoff[it2]) * 2048,
                               (uint32_t)(2048 * ((np2 + 15) & ~15)));
      }
      if (!wait(&bar[kBXready], xpar)) { ok = false; break; }
      xpar ^= 1u;
      const uint64_t dXE0 = tc::smem_desc(xes, tc::kLBO, 16u * (uint32_t)KEp);   // x^E slice j: + j dXEs
      constexpr uint64_t dXEs = (uint64_t)(kXEslice >> 4);
      const uint32_t idT = tc::idesc_bf16(128, KEp > 0 ? KEp : 16);
      const int ns = (np > 0 ? kSlices : 0) + (hasH ? kSlices : 0);
      for (int st = 0; st < ns && ok; ++st) {
        if (*wabort) { ok = false; break; }   // a work warp gave up
        const int slot = (int)(consumed % kNSlot);
        if (!wait(&bar[kBFull0 + slot], (fparb >> slot) & 1u)) { ok = false; break; }
        fparb ^= 1u << slot;
        const bool isE = np > 0 && st < kSlices;
        const int i = isE ? st : (np > 0 ? st - kSlices : st);
        if (!isE && i == 0 && np > 0) {
          // the E pass's classical accumulators must be drained before the H pass reuses them
          if (!wait(&bar[kBDrainedE], dpar)) { ok = false; break; }
          dpar ^= 1u;
        }
        tc::fence_after_sync();
        const uint32_t a = ring + (uint32_t)slot * kSliceBytes;
        if (isE) {
          const uint64_t dEc = tc::smem_desc(a, tc::kLBO, 16u * (uint32_t)KEp);   // E_c slice i (128 x KEp)
          const uint64_t dEt = tc::smem_desc(a + eb, tc::kLBO, 2048);            // E_c^T slice i (KEp x 128)
          for (int j = 0; j < kSlices && i + j <= kMaxGroup; ++j) {
            const int gsum = i + j;
            const uint32_t acc = gsum == 0 ? 0u : gsum == 1 ? 96u : 192u;
            const uint32_t first = (i == 0 && j <= 2) ? 1u : 0u;   // first pair of each accumulator's group
            // E_c x^E: A = E_c slice i, B = x^E slice j (96 x KEp)
            for (int ks = 0; ks < KEp / 16; ++ks)
              tc::mma_bf16_lane0(tm + acc, dEc + 16u * ks, dXE0 + j * dXEs + 16u * ks, idH, (first && ks == 0) ? 0u : 1u);
            // E_c^T x^C: A = x^C slice j (rows n; rows past 96 read the next region and land in
            // tensor-memory lanes that are never read), B = E_c^T slice i
            for (int ks = 0; ks < kK / 16; ++ks)
              tc::mma_bf16_lane0(tm + 288u + acc / 2, dX0 + j * dXs + 16u * ks, dEt + 16u * ks, idT,
                                 (first && ks == 0) ? 0u : 1u);
          }
        } else {
          const uint64_t dH = tc::smem_desc(a, tc::kLBO, 2048);   // H_c slice i (128 x 128)
          for (int j = 0; j < kSlices && i + j <= kMaxGroup; ++j) {
            const int gsum = i + j;
            const uint32_t acc = gsum == 0 ? 0u : gsum == 1 ? 96u : 192u;
            const uint32_t first = (i == 0 && j <= 2) ? 1u : 0u;
            for (int ks = 0; ks < kK / 16; ++ks)
              tc::mma_bf16_lane0(tm + acc, dH + 16u * ks, dX0 + j * dXs + 16u * ks, idH, (first && ks == 0) ? 0u : 1u);
          }
        }
        tc::mma_commit_lane0(&bar[kBEmpty0 + slot]);
        if (isE && st == kSlices - 1) tc::mma_commit_lane0(&bar[kBAccE]);
        ++consumed;
        ok = issue_copy();
      }
      // the work warps' H epilogue waits on this commit also for items without H_c
      if (ok) tc::mma_commit_lane0(&bar[kBAccH]);
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    // nothing may be in flight when the CTA leaves: every copy issued (bounded waits on the ones not
    // consumed) and every MMA (one more commit, on a barrier of its own)
    for (long long s2 = consumed; s2 < issued; ++s2) {
      const int slot = (int)(s2 % kNSlot);
      wait_n(&bar[kBFull0 + slot], (fparb >> slot) & 1u, kWaitLimit);
      fparb ^= 1u << slot;
    }
    tc::mma_commit_lane0(&bar[kBFin]);
    wait_n(&bar[kBFin], 0, kWaitLimit);
  } else {
    // ------------------------------------------------------------ work warps
    uint32_t apar = 0, hpar = 0;
    const int lg = warp & 3, qw = warp >> 2;     // tensor-memory lane quarter, column share (0..kWPQ-1)
    const int r = 32 * lg + lane;                // accumulator row (cell node) of this thread
    const uint32_t lane_addr = (uint32_t)(32 * lg) << 16;
    // warp 0 polls an mbarrier (bounded), the other warps wait at the work barrier; a wait that
    // gave up is recorded before the barrier and read by everyone after it
    auto wait_all = [&](uint64_t* b, uint32_t par) {
      if (warp == 0) {
        const bool okw = __all_sync(0xffffffffu, tc::mbar_wait(b, par, wlim));
        if (!okw && lane == 0) {
          *wabort = 1;
          atomicExch(err, 1);
        }
      }
      tc::named_sync(1, kWork);
      tc::fence_after_sync();
      return *wabort == 0;
    };
    // metadata of cell w into buffer b (every work thread takes part; no barrier inside)
    auto load_meta = [&](long long w, int b) {
      const int item = (int)(w % items.n), m = (int)(w / items.n);
      const int c = items.cell[item];
      const int p0 = items.p0[item], np = items.np[item];
      int cx, cy, cz;
      cell_ijk(mesh, c, cx, cy, cz);
      for (int l = tid; l < 128; l += kWork) {
        if (l < NN)
          gS2[b * 128 + l] = node_index(mesh, cx, cy, cz, l % P1, (l / P1) % P1, l / (P1 * P1)) * ld2 + (long long)m * cols;
        rexpH2[b * 128 + l] = tcRexpH[((long long)m * mesh.nc + c) * 128 + l];
        if (np > 0) rexpE2[b * 128 + l] = tcRexpE[((long long)m * items.n + item) * 128 + l];
      }
      for (int f = tid; f < np; f += kWork) {
        fns2[b * kMaxKE + f] = pair_fn[p0 + f];
        hexp2[b * kMaxKE + f] = tcHexp[(long long)m * n_pairs + p0 + f];
      }
    };
    // gather of x_bar^C (D is folded into the operator): item = (chunk of 8 nodes, column n)
    const int nitem = (kK / 8) * cols;
    double v[kNK][8];
    int buf = 0;
    if ((long long)blockIdx.x < nwork) {
      load_meta(blockIdx.x, 0);
      tc::named_sync(1, kWork);
    }
    for (long long w = blockIdx.x; w < nwork; w += gridDim.x) {
      const int item = (int)(w % items.n), m = (int)(w / items.n);
      const int col0 = m * cols;
      const int np = items.np[item];
      const int iflags = items.flags[item];
      const bool hasH = (iflags & kItemH) != 0, solo = (iflags & kItemSolo) != 0;
      const int KEp = (np + 15) & ~15;
      const long long* gS = gS2 + buf * 128;
      const int* rexpH = rexpH2 + buf * 128;
      const int* rexpE = rexpE2 + buf * 128;
      const int* hexp = hexp2 + buf * kMaxKE;
      const int* fns = fns2 + buf * kMaxKE;
      gather_rows<NN>(X, gS, tid, cols, nitem, v);   // rows prefetched into L2 one cell ahead
      for (int n = tid; n < kMaxN; n += kWork) {
        cmaxC[n] = 0;
        cmaxE[n] = 0;
      }
      tc::named_sync(1, kWork);
      // x^C as float32 pairs (ph, pl); column maxima of |ph|
      float ph[kNK][8], pl[kNK][8];
#pragma unroll
      for (int k = 0; k < kNK; ++k) {
        const int it = tid + k * kWork;
        const int n = it - (it / cols) * cols;
        float mx = 0.0f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const df32 x = split_f64(v[k][t]);
          ph[k][t] = x.h;
          pl[k][t] = x.l;
          mx = fmaxf(mx, fabsf(x.h));
        }
        if (it < nitem && mx > 0.0f) atomicMax(&cmaxC[n], __float_as_int(mx));
      }
      // x^E column maxima (values reloaded for the split below)
      const int nitemE = (KEp / 8) * cols;
      for (int it = tid; it < nitemE; it += kWork) {
        const int ch = it / cols, n = it - ch * cols;
        float mx = 0.0f;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int f = ch * 8 + t;
          if (f < np) mx = fmaxf(mx, fabsf(split_f64(xE[(long long)fns[f] * ld2 + col0 + n]).h));
        }
        if (mx > 0.0f) atomicMax(&cmaxE[n], __float_as_int(mx));
      }
      tc::named_sync(1, kWork);
      for (int n = tid; n < kMaxN; n += kWork) {
        fC[n] = exp_of_maxbits(cmaxC[n]);
        fE[n] = exp_of_maxbits(cmaxE[n]);
      }
      // slices of x^C (rows n, K = node) and of x^E (rows n, K = function)
#pragma unroll
      for (int k = 0; k < kNK; ++k) {
        const int it = tid + k * kWork;
        if (it < nitem) {
          const int ch = it / cols, n = it - ch * cols;
          const int fe = exp_of_maxbits(cmaxC[n]);
          const float sc = fe == kZero ? 0.0f : tc::exp2_neg(fe);
          store_digits8(ph[k], pl[k], sc, sm + kXs + tc::kmajor_offset(n, ch * 8, 2048), kXslice);
        }
      }
      for (int it = tid; it < nitemE; it += kWork) {
        const int ch = it / cols, n = it - ch * cols;
        const int fe = exp_of_maxbits(cmaxE[n]);
        const float sc = fe == kZero ? 0.0f : tc::exp2_neg(fe);
        float a[8], b[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int f = ch * 8 + t;
          const df32 x = f < np ? split_f64(xE[(long long)fns[f] * ld2 + col0 + n]) : df32(0.0f, 0.0f);
          a[t] = x.h;
          b[t] = x.l;
        }
        store_digits8(a, b, sc, sm + kXEs + tc::kmajor_offset(n, ch * 8, 16 * KEp), kXEslice);
      }
      tc::fence_proxy_async();
      tc::named_sync(1, kWork);
      if (tid == 0) tc::mbar_arrive(&bar[kBXready]);
      // while the tensor cores run: the metadata of this CTA's next cell, and its rows of x_bar into
      // L2 (one bulk prefetch per node row)
      const long long wn = w + gridDim.x;
      if (wn < nwork) load_meta(wn, buf ^ 1);
      if (wn < nwork && tid < NN) {
        const long long w2 = wn;
        const int c2 = items.cell[(int)(w2 % items.n)], m2 = (int)(w2 / items.n);
        int ex, ey, ez;
        cell_ijk(mesh, c2, ex, ey, ez);
        const long long g = node_index(mesh, ex, ey, ez, tid % P1, (tid / P1) % P1, tid / (P1 * P1));
        tc::bulk_prefetch_l2(X + g * ld2 + (long long)m2 * cols, (uint32_t)(cols * 8));
      }
      // units of the output (row r, column n): the larger of the units of H_c x^C and E_c x^E;
      // each part is scaled onto them by 2^kH, 2^kE <= 1
      const int reH = r < NN ? rexpH[r] : kZero;
      const int reE = (r < NN && np > 0) ? rexpE[r] : kZero;
      auto down = [](int k) { return k < -125 ? 0.0f : tc::exp2_pos(k); };
      // ---- E pass epilogue: E_c^T x^C to y^E; then E_c x^E as a pair (s, t) in the output's
      // units, parked in tensor-memory columns 288 + 16 ch (s) and 296 + 16 ch (t) of chunk ch
      // (free once E_c^T x^C has been read: the H pass writes columns 0..287 only)
      if (np > 0) {
        const bool okE = wait_all(&bar[kBAccE], apar);
        apar ^= 1u;
        if (okE) {
          // E_c^T x^C: accumulator row = column n of this member, column = function f
          const int n = r;
          const int fe = n < cols ? fC[n] : kZero;
          for (int ch = qw; ch * 8 < KEp; ch += kWPQ) {
            float t0[8], t1[8], t2[8];
            const uint32_t ta = tm + lane_addr + 288 + 8 * ch;
            tc::tmem_ld8x3(ta, ta + 48, ta + 96, t0, t1, t2);
            if (fe != kZero) {
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const int f = 8 * ch + t;
                if (f >= np) break;
                if (hexp[f] == kZero) continue;
                float s, u;
                tc::sum3_pair(t0[t], t1[t], t2[t], s, u);
                if (s != 0.0f) atomicAdd(&yE[(long long)fns[f] * ld2 + col0 + n], tc::double_of_pair(s, u, fe + hexp[f]));
              }
            }
          }
        }
        tc::fence_before_sync();
        tc::named_sync(1, kWork);   // every warp has read E_c^T x^C before its columns are reused
        tc::fence_after_sync();
        if (okE) {
#pragma unroll
          for (int q = 0; q < kNQ; ++q) {
            const int ch = qw + kWPQ * q;
            if (ch * 8 < nm) {
              float a0[8], a1[8], a2[8], sE[8], tE[8];
              const uint32_t t0 = tm + lane_addr + 8 * ch;
              tc::tmem_ld8x3(t0, t0 + 96, t0 + 192, a0, a1, a2);
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const int n = 8 * ch + t;
                const int eH = (!hasH || reH == kZero || fC[n] == kZero) ? kZero : reH + fC[n];
                const int eE = (reE == kZero || fE[n] == kZero) ? kZero : reE + fE[n];
                float s, u;
                tc::sum3_pair(a0[t], a1[t], a2[t], s, u);
                const float sc = eE == kZero ? 0.0f : down(eE - (eH > eE ? eH : eE));
                sE[t] = __fmul_rn(s, sc);
                tE[t] = __fmul_rn(u, sc);
              }
              tc::tmem_st8x2(tm + lane_addr + 288 + 16 * ch, tm + lane_addr + 296 + 16 * ch, sE, tE);
            }
          }
        }
        tc::fence_before_sync();
        tc::named_sync(1, kWork);
        // the issuer waits for this only before an H pass (items that carry H_c): one arrival per wait
        if (tid == 0 && hasH) tc::mbar_arrive(&bar[kBDrainedE]);
        if (*wabort) break;
      }
      // ---- H pass epilogue: H_c x^C (+ the E part) -> y_c (staged in shared memory)
      const bool okH = wait_all(&bar[kBAccH], hpar);
      hpar ^= 1u;
      if (okH) {
#pragma unroll
        for (int q = 0; q < kNQ; ++q) {
          const int ch = qw + kWPQ * q;
          if (ch * 8 < nm) {
            float a0[8], a1[8], a2[8], sE[8], tE[8];
            const uint32_t t0 = tm + lane_addr + 8 * ch;
            if (hasH) {
              tc::tmem_ld8x3(t0, t0 + 96, t0 + 192, a0, a1, a2);
            } else {
#pragma unroll
              for (int t = 0; t < 8; ++t) a0[t] = a1[t] = a2[t] = 0.0f;
            }
            if (np > 0) tc::tmem_ld8x2(tm + lane_addr + 288 + 16 * ch, tm + lane_addr + 296 + 16 * ch, sE, tE);
            if (r < NN) {
#pragma unroll
              for (int t = 0; t < 8; ++t) {
                const int n = 8 * ch + t;
                if (n < cols) {
                  const int eH = (!hasH || reH == kZero || fC[n] == kZero) ? kZero : reH + fC[n];
                  double y = 0.0;
                  float s, u;
                  if (np == 0) {
                    if (eH != kZero) {
                      tc::sum3_pair(a0[t], a1[t], a2[t], s, u);
                      y = tc::double_of_pair(s, u, eH);
                    }
                  } else {
                    const int eE = (reE == kZero || fE[n] == kZero) ? kZero : reE + fE[n];
                    const int eO = eH > eE ? eH : eE;
                    if (eO != kZero) {
                      const float sc = eH == kZero ? 0.0f : down(eH - eO);
                      tc::sum5_pair(__fmul_rn(a0[t], sc), __fmul_rn(a1[t], sc), __fmul_rn(a2[t], sc), sE[t], tE[t],
                                    s, u);
                      y = tc::double_of_pair(s, u, eO);
                    }
                  }
                  stage[r * kStageLd + n] = y;
                }
              }
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::named_sync(1, kWork);
      if (*wabort) break;
      // scatter: one node row per warp, consecutive columns per lane
      for (int l = warp; l < NN; l += kWork / 32) {
        const int a = l % P1, b = (l / P1) % P1, cc = l / (P1 * P1);
        const bool interior = solo && a > 0 && a < P1 - 1 && b > 0 && b < P1 - 1 && cc > 0 && cc < P1 - 1;
        double* yrow = Y + gS[l];
        for (int n = lane; n < cols; n += 32) {
          const double y = stage[l * kStageLd + n];
          if (interior)
            yrow[n] = y;
          else if ((__double_as_longlong(y) << 1) != 0)
            atomicAdd(&yrow[n], y);
        }
      }
      tc::named_sync(1, kWork);   // staging (the x^C slices) free for the next cell
      buf ^= 1;
    }
  }
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
  // one member: the apply runs over blocks of 96 real columns; several members: one block each
  if (c.batch > 1 && cols_member > kMaxN)
    return "EFE_TC needs at most 96 real columns (48 orbitals) per batch member when batch > 1";
  return nullptr;
}

static TcItems tc_items(const Ctx& c) {
  const TcState& t = c.tc;
  return TcItems{t.n_items, t.items, t.items + t.n_items, t.items + 2 * t.n_items, t.items + 3 * t.n_items, t.eoff,
                 t.first_item};
}

static cudaError_t tc_alloc(Ctx& c, int batch) {
  TcState& t = c.tc;
  if (t.eoff == nullptr) {
    std::vector<int> ps(c.nc + 1, 0);
    if (c.n_pairs > 0)
      EFE_CUDA_TRY(cudaMemcpy(ps.data(), c.d_pair_start, sizeof(int) * (c.nc + 1), cudaMemcpyDeviceToHost));
    // work items: a cell's pairs in runs of at most kMaxKE; the first item of a cell carries H_c
    std::vector<int> cell, p0, np, flags, first(c.nc + 1, 0);
    for (int i = 0; i < c.nc; ++i) {
      first[i] = (int)cell.size();
      const int n = ps[i + 1] - ps[i];
      const int k = n > 0 ? (n + kMaxKE - 1) / kMaxKE : 1;
      for (int q = 0; q < k; ++q) {
        cell.push_back(i);
        p0.push_back(ps[i] + q * kMaxKE);
        np.push_back(std::min(kMaxKE, n - q * kMaxKE) > 0 ? std::min(kMaxKE, n - q * kMaxKE) : 0);
        flags.push_back((q == 0 ? kItemH : 0) | (k == 1 ? kItemSolo : 0));
      }
    }
    first[c.nc] = (int)cell.size();
    t.n_items = (int)cell.size();
    std::vector<int> packed;
    packed.reserve(4 * (size_t)t.n_items);
    for (auto* v : {&cell, &p0, &np, &flags}) packed.insert(packed.end(), v->begin(), v->end());
    std::vector<long long> eo(t.n_items + 1, 0);
    for (int i = 0; i < t.n_items; ++i) eo[i + 1] = eo[i] + ((np[i] + 15) & ~15);
    t.e_total = eo[t.n_items];
    EFE_CUDA_TRY(cudaMalloc(&t.items, sizeof(int) * packed.size()));
    EFE_CUDA_TRY(cudaMemcpy(t.items, packed.data(), sizeof(int) * packed.size(), cudaMemcpyHostToDevice));
    EFE_CUDA_TRY(cudaMalloc(&t.first_item, sizeof(int) * (c.nc + 1)));
    EFE_CUDA_TRY(cudaMemcpy(t.first_item, first.data(), sizeof(int) * (c.nc + 1), cudaMemcpyHostToDevice));
    EFE_CUDA_TRY(cudaMalloc(&t.eoff, sizeof(long long) * (t.n_items + 1)));
    EFE_CUDA_TRY(cudaMemcpy(t.eoff, eo.data(), sizeof(long long) * (t.n_items + 1), cudaMemcpyHostToDevice));
    EFE_CUDA_TRY(cudaMalloc(&t.err, sizeof(int)));
    EFE_CUDA_TRY(cudaMemset(t.err, 0, sizeof(int)));
  }
  if (t.batch != batch) {
    cudaFree(t.H); cudaFree(t.rexp); cudaFree(t.rexpE); cudaFree(t.E); cudaFree(t.hexp);
    t.H = nullptr; t.rexp = nullptr; t.rexpE = nullptr; t.E = nullptr; t.hexp = nullptr;
    t.batch = 0;
    EFE_CUDA_TRY(cudaMalloc(&t.H, (size_t)batch * c.nc * kSlices * kSliceBytes));
    EFE_CUDA_TRY(cudaMalloc(&t.rexp, sizeof(int) * (size_t)batch * c.nc * 128));
    EFE_CUDA_TRY(cudaMalloc(&t.rexpE, sizeof(int) * (size_t)batch * t.n_items * 128));
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
  const size_t sm = sizeof(double) * (S3 + PP * NQ1 + PP * NQ1 * NQ1 + PP * PP * NQ1 + NN * NN + 128) +
                    sizeof(int) * (128 + 128 + 48);
  auto f = k_tc_build<P1, NQ1>;
  EFE_CUDA_TRY(set_smem_tc(f, sm));
  dim3 grid(c.nc, batch);
  f<<<grid, 256, sm, s>>>(c.tab, c.mesh, c.op.W64, c.op.kin, c.n_pairs > 0 ? c.d_pair_start : nullptr, c.op.E64,
                          c.n_pairs, c.d_Dsc, tc_items(c), c.tc.e_total, c.tc.H, c.tc.rexp, c.tc.rexpE, c.tc.E,
                          c.tc.hexp);
  note_launch();
  return cudaGetLastError();
}

template <int P1>
static cudaError_t tc_apply_impl(Ctx& c, const double* X, double* Y, long long n_cols, long long ld, cudaStream_t s) {
  const long long ld2 = 2 * ld;
  const int batch = c.op.batch;
  const int cols_all = (int)(2 * n_cols / batch);
  const int ncols2 = (int)(2 * n_cols);
  EFE_CUDA_TRY(cudaMemset2DAsync(Y, sizeof(double) * ld2, 0, sizeof(double) * ncols2, c.n_dof, s));
  if (c.nE > 0) {
    EFE_CUDA_TRY(cudaMemsetAsync(c.d_yE, 0, sizeof(double) * c.nE * ld2, s));
    EFE_CUDA_TRY(launch_enr_pre(c, X, ld2, ncols2, s));
  }
  if (c.tc.n_sm == 0) EFE_CUDA_TRY(cudaDeviceGetAttribute(&c.tc.n_sm, cudaDevAttrMultiProcessorCount, c.device));
  const long long nwork = (long long)c.tc.n_items * batch;
  const unsigned grid = (unsigned)(nwork < c.tc.n_sm ? nwork : c.tc.n_sm);
  auto f = k_tc_apply<P1>;
  EFE_CUDA_TRY(set_smem_tc(f, kApplySmem));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!c.apply_gate) prof_pair(c, e0, e1);
  if (e0) EFE_CUDA_TRY(cudaEventRecord(e0, s));
  // one member: blocks of at most 96 real columns (one launch each); several members: one launch
  const int blk = batch == 1 ? kMaxN : cols_all;
  for (int off = 0; off < cols_all; off += blk) {
    const int cols = std::min(blk, cols_all - off);
    const int nm = (cols + 15) & ~15;
    f<<<grid, kApplyThreads, kApplySmem, s>>>(c.mesh, X + off, Y + off, ld2, cols, nm, batch, c.d_Dsc, c.tc.H,
                                              c.tc.rexp, c.tc.rexpE, c.tc.E, c.tc.e_total, tc_items(c), c.tc.hexp,
                                              c.d_pair_fn, c.n_pairs, c.d_xE + off, c.d_yE + off, c.tc.err,
                                              c.apply_gate, c.tc_wait_limit > 0 ? c.tc_wait_limit : kWaitLimit);
    note_launch();
    EFE_CUDA_TRY(cudaGetLastError());
  }
  if (e1) EFE_CUDA_TRY(cudaEventRecord(e1, s));
  if (c.nE > 0) EFE_CUDA_TRY(launch_enr_post(c, Y, ld2, ncols2, cols_all, s));
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
  cudaFree(t.H); cudaFree(t.rexp); cudaFree(t.rexpE); cudaFree(t.E); cudaFree(t.hexp); cudaFree(t.eoff);
  cudaFree(t.items); cudaFree(t.first_item); cudaFree(t.err);
  t = TcState{};
}

}  // namespace efe
