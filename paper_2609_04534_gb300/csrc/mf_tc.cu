// mf_tc.cu -- the FP64 Cartesian apply on the tensor cores (tcgen05), for degrees 1..3.
//
// On an axis-aligned uniform mesh every cell has the same element matrix
//   A_e = gx K(x)M(x)M + gy M(x)K(x)M + gz M(x)M(x)K [+ c M(x)M(x)M]
// (Sec. 3.1, Eq. (eval_pipeline), Kronecker factors z, y, x), so the local apply of a group
// of cells is one dense product Y[cells, n^3] = X[cells, n^3] A_e^T.  GB300 has no fast FP64
// tensor path, so the product is made exact on the FP16 tensor cores by splitting both
// operands into integer digits (the error-free splitting of the Ozaki scheme: Ozaki, Ogita,
// Oishi, Rump, "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59 (2012)):
//
//  - data: per cell c, E_c is the exponent with |x_j| < 2^E_c for all its values; each value
//    becomes the 48-bit integer X_j = round(x_j 2^(47 - E_c)), written in six balanced base-256
//    digits d_a (a = 0 most significant; d_0 in [-128, 128], the others in [-128, 127]):
//    x_j = sum_a d_a 2^(E_c - 7 - 8a) up to 2^-48 of the cell's largest value;
//  - table: per output row i, F_i with |A_ij| < 2^F_i, and six digits t_b the same way;
//  - level t = a + b collects sum_{a+b=t} sum_j d_a t_b: integers with |.| <= 6 n^3 2^14
//    (2^22.6 at n = 4), so the FP32 accumulator of the tensor core holds every partial sum
//    exactly; levels t > 5 (below 2^-48 of the leading term) are dropped;
//  - y_i = 2^(E_c + F_i - 54) sum_t C_t 256^(5 - t), combined in 64-bit integers and rounded
//    once to double.
//
// Result: within a few 2^-48 of |A_e| |x| per value (rounding of both operands, the dropped
// levels), the accuracy class of the double-float path, and no FP64 or FP32 arithmetic in the
// contraction.  The 21 digit products of a
// group (M = 128 cells = 4 native tiles, N = K = n^3 padded to a multiple of 16) run as
// tcgen05.mma kind::f16 with FP32 accumulators in tensor memory (6 levels x N columns);
// operands sit in shared memory in the K-major, non-swizzled canonical layout.
//
// Kernel structure (persistent, one CTA of 512 threads per SM): thread (cell c, quarter q)
// holds a quarter of its cell's values and combines a quarter of its outputs; per group it
// (1) waits for the previous group's products, reads that group's six levels from tensor
// memory, combines and stores them, (2) reads its quarter of the group's x from shared memory
// (a bulk copy that thread 0 started one group earlier) and writes its largest exponent,
// (3) writes its digits, and (4) thread 0 issues the products: per data digit a one MMA per
// 256 columns against the concatenated table digits [T_0 | ... | T_(5-a)], which puts level
// a + b in its own TMEM columns (32 instructions at n = 4).  Every wait on an mbarrier is
// bounded; on expiry the kernel records an error (mf_device_error) and leaves, freeing its
// tensor memory.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>

#include "mf_kernels.cuh"

namespace mf {
namespace {

constexpr int TC_S = 6;     // digits per value (data and table) and levels kept
constexpr int TC_M = 128;   // cells per group: 4 native tiles, one TMEM lane each
constexpr int TC_NT = 512;  // threads: four per cell (a quarter of its values and outputs each)
constexpr long long TC_WAIT_LIMIT = 1LL << 26; // mbarrier polls before giving up

__device__ int g_tc_error; // nonzero: a bounded wait gave up (read by mf_device_error)

template <int N>
struct TcCfg {
  static constexpr int NN = N * N * N;
  static constexpr int KP = (NN + 15) / 16 * 16;      // K = N of the MMA (padded)
  static constexpr int VPT = KP / 4;                   // values (and outputs) per thread
  static constexpr int CH = VPT < 8 ? VPT : 8;         // values per shared-memory store / TMEM load
  static constexpr int ACC = TC_S * KP;                // TMEM columns of the levels
  static constexpr int TMEM = ACC <= 32 ? 32 : ACC <= 64 ? 64 : ACC <= 128 ? 128 : ACC <= 256 ? 256 : 512;
  static constexpr int A_SLICE = TC_M * KP * 2;        // bytes of one digit slice of the data
  static constexpr int B_SLICE = KP * KP * 2;          // bytes of one digit slice of the table
  static constexpr int X_BYTES = 4 * NN * BL * 8;      // the group's x (4 tiles), staged by TMA
  static constexpr int SMEM_USED = TC_S * (A_SLICE + B_SLICE) + X_BYTES;
  // one CTA per SM: request more than half of the SM's 228 KB so that a second CTA never
  // shares the SM (its tensor-memory allocation could otherwise wait on this one)
  static constexpr int SMEM = SMEM_USED > 117 * 1024 ? SMEM_USED : 117 * 1024;
  static_assert(NN <= 64, "the tensor-core apply covers n <= 4");
  static_assert(VPT % 4 == 0, "stores of at least 4 values");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Byte offset of (row r, k) in a K-major, non-swizzled UMMA operand with kk columns: 8x16-byte
// core matrices, adjacent along K at 128 B (LBO), 8-row groups at kk * 16 B (SBO).
__host__ __device__ __forceinline__ uint32_t kmaj_off(int r, int k, int kk) {
  return (uint32_t)((r >> 3) * (kk * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start, LBO, SBO (all >> 4), version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
  for (long long i = 0; i < TC_WAIT_LIMIT; ++i) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(addr), "r"(parity)
                 : "memory");
    if (ok) return true;
  }
  return false;
}

struct TcArgs {
  const double* x;   // 16-byte aligned (checked on the host)
  double* y;
  const uint4* btab; // TC_S table digit slices in the canonical operand layout
  GridInfo g;
  long long ngroups;
  int fexp[64];      // F_i + 1023 (biased), per output row
};

// Thread 0: the bulk copy of group grp's x (its real tiles, contiguous in the native layout)
// into the staging buffer, completing on mbarrier xbar.
template <int N>
__device__ __forceinline__ void tc_stage_x(const TcArgs& a, long long grp, void* stage, uint32_t xbar) {
  using C = TcCfg<N>;
  const long long t0 = grp * 4;
  const long long nt = a.g.ntiles - t0 < 4 ? a.g.ntiles - t0 : 4;
  const uint32_t bytes = (uint32_t)(nt * C::NN * BL * 8);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(xbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(stage)),
               "l"(a.x + t0 * C::NN * BL), "r"(bytes), "r"(xbar)
               : "memory");
}

// Two values' digits of slice a packed as half2 (low half: value xl).  Digit a of the offset
// integer To = X + 0x808080808080 (0 <= To < 2^48 + 2^40) is u - 128 with u = byte 5 - a of
// To for a > 0 (u in [0, 255]) and u = To >> 40 for a = 0 (u in [0, 256]: the carry of a value
// rounded up to its cell's power of two lands there, so the top digit spans [-128, 128]).  The
// half with bits 0x6400 | u is 1024 + u, and subtracting 1152 leaves the digit exactly.
__device__ __forceinline__ uint32_t digit_pair(uint64_t xl, uint64_t xr, int a) {
  uint32_t w;
  if (a == 0) {
    const uint32_t ul = (uint32_t)(xl >> 40), ur = (uint32_t)(xr >> 40);
    w = ul | (ur << 16) | 0x64006400u;
  } else {
    const int byte = 5 - a;
    const uint32_t wl = byte >= 4 ? (uint32_t)(xl >> 32) : (uint32_t)xl;
    const uint32_t wr = byte >= 4 ? (uint32_t)(xr >> 32) : (uint32_t)xr;
    const uint32_t b = (uint32_t)(byte & 3);
    const uint32_t sel = b | ((b + 4u) << 8);    // byte b of wl -> byte 0, of wr -> byte 2
    w = (__byte_perm(wl, wr, sel) & 0x00ff00ffu) | 0x64006400u;
  }
  __half2 h = *reinterpret_cast<__half2*>(&w);
  h = __hsub2(h, __halves2half2(__ushort_as_half((unsigned short)0x6480), __ushort_as_half((unsigned short)0x6480)));
  return *reinterpret_cast<uint32_t*>(&h);
}

// The offset integer X + 0x808080808080 of x relative to the cell exponent emax (biased):
// X = round(|x| 2^(1069 - emax)) (half up, |X| <= 2^47) with the sign of x; zero, subnormal
// and values more than 48 binades below emax give X = 0.
__device__ __forceinline__ uint64_t fixed_offset(double x, int emax) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int eb = (int)(bits >> 52) & 0x7ff;
  const int sh = 5 + (emax - eb); // one bit more than the target, for the rounding
  unsigned long long X = 0;
  if (eb != 0 && sh < 60) X = ((((bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) >> sh) + 1ull) >> 1;
  const unsigned long long neg = (unsigned long long)((long long)bits >> 63); // 0 or all ones
  return ((X ^ neg) - neg) + 0x808080808080ull;
}

// An exact integer held in a float (|v| <= 2^22) as int: two full-rate instructions.
__device__ __forceinline__ int small_float_int(float v) {
  return __float_as_int(v + 12582912.0f) - 0x4B400000;
}

// double nearest below |Y| 2^p with the sign of Y (truncated: the value already carries the
// ~2^-48 error of the digit products); 0 for Y = 0; underflow to 0, overflow to inf.
__device__ __forceinline__ double scaled_to_double(long long Y, int p) {
  const unsigned long long neg = (unsigned long long)(Y >> 63);
  unsigned long long U = ((unsigned long long)Y ^ neg) - neg;
  const int lz = __clzll(U);                 // 64 for U = 0
  U <<= (lz & 63);                           // leading one at bit 63
  const int e = p + 1086 - lz;               // Y 2^p = (U >> 11) 2^(e - 1075)
  unsigned long long bits = (neg << 63) | ((unsigned long long)(unsigned)e << 52) + ((U >> 11) & 0xFFFFFFFFFFFFFull);
  if ((unsigned)(e - 1) >= 2046u || U == 0) // rare: zero, underflow or overflow
    bits = (neg << 63) | (U == 0 || e <= 0 ? 0ull : 0x7FF0000000000000ull);
  return __longlong_as_double((long long)bits);
}

// The tile and cell coordinates of cell c of group grp; valid = a real cell of the mesh.
__device__ __forceinline__ bool tc_cell(const GridInfo& g, long long grp, int c, long long& t, int& cx, int& cy,
                                        int& cz) {
  t = grp * 4 + (c >> 5);
  cx = cy = cz = 0;
  if (t >= g.ntiles) return false;
  cell_of(g, t, c & 31, cx, cy, cz);
  return cx < g.nx && cy < g.ny && cz < g.nz;
}

template <int N>
__global__ void __launch_bounds__(TC_NT, 1) apply_cartesian_tc(const __grid_constant__ TcArgs a) {
  using C = TcCfg<N>;
  constexpr int NN = C::NN, KP = C::KP, VPT = C::VPT, CH = C::CH;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* sA = tc_smem;                        // TC_S slices [128 cells x KP]
  unsigned char* sB = tc_smem + TC_S * C::A_SLICE;    // [T_0 | ... | T_5]: TC_S * KP rows x KP
  double* sX = reinterpret_cast<double*>(sB + TC_S * C::B_SLICE); // the group's x, native layout
  __shared__ __align__(8) unsigned long long mbar, xbar;
  __shared__ uint32_t tslot;
  __shared__ int emax_s[4][TC_M];                     // [quarter][cell] of the current group
  __shared__ int emc_s[2][TC_M];                      // [group parity][cell]: the cell's exponent
  const int tid = threadIdx.x, warp = tid >> 5;
  const int c = (warp & 3) * 32 + (tid & 31), q = warp >> 2;

  // the table digits (identical for every CTA): global -> shared, once
  for (int i = tid; i < TC_S * C::B_SLICE / 16; i += TC_NT) reinterpret_cast<uint4*>(sB)[i] = a.btab[i];
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&xbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tslot)),
                 "r"(C::TMEM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = tslot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t xbar_a = smem_addr(&xbar), mbar_a = smem_addr(&mbar);
  long long g = blockIdx.x;
  if (tid == 0) tc_stage_x<N>(a, g, sX, xbar_a); // the grid never exceeds the number of groups

  // Combine the six levels of group gp (cell exponent emc) for CH of this thread's outputs
  // from i0: Y = sum_t C_t 256^(5-t) in 64-bit integers (C_0 256 + C_1 fills the high word),
  // y = Y 2^(E_c + F_i - 54); stores them (0 for padding cells of real tiles, nothing for
  // missing tiles).
  auto combine = [&](long long gp, int emc, int i0) {
    long long t;
    int cx, cy, cz;
    const bool valid = tc_cell(a.g, gp, c, t, cx, cy, cz);
    double* __restrict__ yp = a.y + t * (long long)NN * BL + (c & 31);
    {
      uint32_t r[TC_S][CH];
#pragma unroll
      for (int lv = 0; lv < TC_S; ++lv) {
        const uint32_t ta = tbase + lane_base + (uint32_t)(lv * KP + i0);
        if constexpr (CH == 8)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                       : "=r"(r[lv][0]), "=r"(r[lv][1]), "=r"(r[lv][2]), "=r"(r[lv][3]), "=r"(r[lv][4]),
                         "=r"(r[lv][5]), "=r"(r[lv][6]), "=r"(r[lv][7])
                       : "r"(ta));
        else
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                       : "=r"(r[lv][0]), "=r"(r[lv][1]), "=r"(r[lv][2]), "=r"(r[lv][3])
                       : "r"(ta));
      }
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (t >= a.g.ntiles) return;
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int i = i0 + j;
        if (i >= NN) continue;
        double yv = 0.0;
        if (valid) {
          // |C_0..C_3| <= 4 n^3 2^14 <= 2^22; C_4, C_5 up to 6 n^3 2^14 take the conversion unit
          const int c0 = small_float_int(__uint_as_float(r[0][j]));
          const int c1 = small_float_int(__uint_as_float(r[1][j]));
          const int c2 = small_float_int(__uint_as_float(r[2][j]));
          const int c3 = small_float_int(__uint_as_float(r[3][j]));
          const int c4 = __float2int_rn(__uint_as_float(r[4][j]));
          const int c5 = __float2int_rn(__uint_as_float(r[5][j]));
          const long long L = (long long)c5 + (long long)c4 * 256LL + (long long)c3 * 65536LL + (long long)c2 * 16777216LL;
          const long long Y = (long long)((unsigned long long)(long long)(c0 * 256 + c1) << 32) + L;
          yv = emc == 2047 ? __longlong_as_double(0x7FF8000000000000LL) // a non-finite input
                           : scaled_to_double(Y, emc + a.fexp[i] - 2099);  // 2^(E_c + F_i - 54)
          if (a.g.bc && on_cube_boundary<N>(a.g, cx, cy, cz, i % N, (i / N) % N, i / (N * N))) yv = 0.0;
        }
        yp[(long long)i * BL] = yv;
      }
    }
  };

  long long gprev = -1;
  int it = 0;
  int abort_all = 0;
  for (; g < a.ngroups; g += gridDim.x, ++it) {
    // (1) this group's x from the staging buffer (copied one phase earlier), masked, and its
    // quarter's largest biased exponent (2047 marks a non-finite value); the previous group's
    // products are still running meanwhile
    int bad = !mbar_wait(xbar_a, (uint32_t)(it & 1));
    double xv[VPT];
    {
      long long t;
      int cx, cy, cz;
      const bool valid = tc_cell(a.g, g, c, t, cx, cy, cz);
      const double* xs = sX + (long long)(c >> 5) * NN * BL + (c & 31);
#pragma unroll
      for (int j = 0; j < VPT; ++j) {
        const int l = q * VPT + j;
        double v = 0.0;
        if (valid && l < NN) {
          v = xs[l * BL];
          if (a.g.bc && on_cube_boundary<N>(a.g, cx, cy, cz, l % N, (l / N) % N, l / (N * N))) v = 0.0;
        }
        xv[j] = v;
      }
    }
    int em = 0;
#pragma unroll
    for (int j = 0; j < VPT; ++j) em = max(em, (int)((unsigned long long)__double_as_longlong(xv[j]) >> 52) & 0x7ff);
    emax_s[q][c] = em;
    abort_all = __syncthreads_or(bad);
    if (abort_all) break;
    // the staging buffer is free: thread 0 starts the next group's copy (after the barrier,
    // ordered behind every thread's reads of the buffer)
    if (tid == 0 && g + gridDim.x < a.ngroups) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_stage_x<N>(a, g + gridDim.x, sX, xbar_a);
    }
    const int emc = max(max(emax_s[0][c], emax_s[1][c]), max(emax_s[2][c], emax_s[3][c]));
    if (q == 0) emc_s[it & 1][c] = emc;
    // (2) the previous group's products; the tensor memory and the digit buffer are free
    // once they have landed
    if (it > 0) {
      bad = !mbar_wait(mbar_a, (uint32_t)((it - 1) & 1));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      abort_all = __syncthreads_or(bad);
      if (abort_all) break;
    }
    // (3) chunk by chunk: combine and store CH outputs of the previous group, and write the
    // digits of CH values of this group (two independent instruction streams per thread)
    const int emp = it > 0 ? emc_s[(it - 1) & 1][c] : 0;
#pragma unroll
    for (int k0 = 0; k0 < VPT; k0 += CH) {
      if (it > 0) combine(gprev, emp, q * VPT + k0);
      uint64_t X[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) X[j] = fixed_offset(xv[k0 + j], emc);
      const uint32_t off = kmaj_off(c, q * VPT + k0, KP);
#pragma unroll
      for (int sl = 0; sl < TC_S; ++sl) {
        if constexpr (CH == 8) {
          uint4 w;
          w.x = digit_pair(X[0], X[1], sl);
          w.y = digit_pair(X[2], X[3], sl);
          w.z = digit_pair(X[4], X[5], sl);
          w.w = digit_pair(X[6], X[7], sl);
          *reinterpret_cast<uint4*>(sA + sl * C::A_SLICE + off) = w;
        } else {
          uint2 w;
          w.x = digit_pair(X[0], X[1], sl);
          w.y = digit_pair(X[2], X[3], sl);
          *reinterpret_cast<uint2*>(sA + sl * C::A_SLICE + off) = w;
        }
      }
    }
    gprev = g;
    // (4) digits visible to the tensor cores; thread 0 issues, per data digit a, the products
    // with all table digits b <= 5 - a at once: D[:, a KP ...] += X_a [T_0 | ... | T_(5-a)]
    // (level a + b lands in TMEM columns (a + b) KP), in chunks of at most 256 columns
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t a0 = umma_desc(smem_addr(sA), 128, KP * 16);
      const uint64_t b0 = umma_desc(smem_addr(sB), 128, KP * 16);
#pragma unroll
      for (int da = 0; da < TC_S; ++da) {
#pragma unroll
        for (int c0 = 0; c0 < (TC_S - da) * KP; c0 += 256) {
          const int nb = (TC_S - da) * KP - c0 < 256 ? (TC_S - da) * KP - c0 : 256;
          const uint32_t idesc = (1u << 4) | ((uint32_t)(nb >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
#pragma unroll
          for (int ks = 0; ks < KP / 16; ++ks) {
            // descriptor addresses advance in 16-byte units: slice da, B row c0, k-step ks
            const uint64_t ad = a0 + (uint64_t)((da * C::A_SLICE + ks * 256) >> 4);
            const uint64_t bd = b0 + (uint64_t)(((c0 / 8) * KP * 16 + ks * 256) >> 4);
            const uint32_t acc = (da > 0 || ks > 0) ? 1u : 0u;
            asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %4, 0;\n"
                         " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n}\n" ::"r"(
                             tbase + (uint32_t)(da * KP + c0)),
                         "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                   : "memory");
    }
  }
  // the last group
  if (!abort_all && it > 0) {
    const int bad = !mbar_wait(mbar_a, (uint32_t)((it - 1) & 1));
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!bad)
#pragma unroll
      for (int i0 = q * VPT; i0 < (q + 1) * VPT; i0 += CH) combine(gprev, emc_s[(it - 1) & 1][c], i0);
    abort_all = __syncthreads_or(bad);
  }
  if (abort_all) {
    if (tid == 0) atomicExch(&g_tc_error, 1);
    // give copies and products still in flight a bounded time to land before the memory is
    // freed: the staged copy of the group the loop stopped at, and the last products
    mbar_wait(xbar_a, (uint32_t)(it & 1));
    if (it > 0) mbar_wait(mbar_a, (uint32_t)((it - 1) & 1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(C::TMEM));
}

// ---------------------------------------------------------------------------------------
// Host: the digit table of the element matrix and the launch.
// ---------------------------------------------------------------------------------------
template <int N>
size_t tc_table_bytes_n() {
  return (size_t)TC_S * TcCfg<N>::B_SLICE;
}

// Element matrix (long double), per-row exponents and the digit slices in operand layout.
template <int N>
void tc_make_table(const mf_operator* op, std::vector<unsigned short>& half_bits, int* fexp) {
  using C = TcCfg<N>;
  constexpr int NN = C::NN, KP = C::KP;
  const HostTables& tb = op->tab;
  auto M1 = [&](int i, int j) { return (long double)tb.M[i * MAXN + j]; };
  auto K1 = [&](int i, int j) { return (long double)tb.K[i * MAXN + j]; };
  std::vector<long double> A((size_t)NN * NN);
  for (int i = 0; i < NN; ++i) {
    const int ix = i % N, iy = (i / N) % N, iz = i / (N * N);
    for (int j = 0; j < NN; ++j) {
      const int jx = j % N, jy = (j / N) % N, jz = j / (N * N);
      const long double mx = M1(ix, jx), my = M1(iy, jy), mz = M1(iz, jz);
      A[(size_t)i * NN + j] = (long double)op->gx * K1(ix, jx) * my * mz + (long double)op->gy * mx * K1(iy, jy) * mz +
                              (long double)op->gz * mx * my * K1(iz, jz) + (long double)op->cmass * mx * my * mz;
    }
  }
  half_bits.assign((size_t)TC_S * KP * KP, 0);
  for (int i = 0; i < 64; ++i) fexp[i] = 0;
  for (int i = 0; i < NN; ++i) {
    long double amax = 0.0L;
    for (int j = 0; j < NN; ++j) amax = std::fmax(amax, std::fabs(A[(size_t)i * NN + j]));
    int F = 0;
    if (amax > 0.0L) {
      std::frexp(amax, &F); // amax = f 2^F, f in [0.5, 1): |A_ij| < 2^F
    } else {
      F = -1000;
    }
    fexp[i] = F + 1023;
    for (int j = 0; j < NN; ++j) {
      long long T = std::llround(std::ldexp(A[(size_t)i * NN + j], 47 - F)); // |T| <= 2^47
      if (amax == 0.0L) T = 0;
      const unsigned long long To = (unsigned long long)(T + 0x808080808080LL);
      for (int b = 0; b < TC_S; ++b) {
        // the top digit keeps its carry (u up to 256), the others are bytes
        const int u = b == 0 ? (int)(To >> 40) : (int)((To >> (8 * (5 - b))) & 0xff);
        const __half hv = __float2half_rn((float)(u - 128));
        unsigned short bits;
        std::memcpy(&bits, &hv, 2);
        half_bits[((size_t)b * C::B_SLICE + kmaj_off(i, j, KP)) / 2] = bits;
      }
    }
    // padded K columns (j >= NN) keep the digit 0 (bits 0)
  }
}

int g_sms = 0;
std::mutex g_sms_mu;
int sm_count() {
  std::lock_guard<std::mutex> lk(g_sms_mu);
  if (g_sms == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    g_sms = v > 0 ? v : 1;
  }
  return g_sms;
}

template <int N>
mf_status tc_launch_n(const mf_operator* op, const void* x, void* y, cudaStream_t s) {
  using C = TcCfg<N>;
  TcArgs a;
  a.x = static_cast<const double*>(x);
  a.y = static_cast<double*>(y);
  a.btab = static_cast<const uint4*>(op->tc_table);
  a.g = op->g;
  a.ngroups = (op->g.ntiles + 3) / 4;
  for (int i = 0; i < 64; ++i) a.fexp[i] = op->tc_fexp[i];
  if (a.ngroups <= 0) return MF_OK;
  if (reinterpret_cast<uintptr_t>(x) & 15)
    return set_error(MF_ERR_ARG, "tensor-core apply: x must be 16-byte aligned");
  static bool attr_set = false; // per degree (template instance)
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(apply_cartesian_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (e != cudaSuccess) return cuda_check(e, "cudaFuncSetAttribute(tensor-core apply)");
    attr_set = true;
  }
  long long grid = (long long)sm_count();
  if (grid > a.ngroups) grid = a.ngroups;
  apply_cartesian_tc<N><<<(unsigned)grid, TC_NT, C::SMEM, s>>>(a);
  return cuda_check(cudaGetLastError(), "tensor-core apply launch");
}

} // namespace

bool tc_eligible(const mf_operator* op) {
  return op->path == PATH_CARTESIAN && op->precision == MF_FP64 && op->n >= 2 && op->n <= 4;
}

size_t tc_table_bytes(const mf_operator* op) {
  if (!tc_eligible(op)) return 0;
  switch (op->n) {
    case 2: return tc_table_bytes_n<2>();
    case 3: return tc_table_bytes_n<3>();
    default: return tc_table_bytes_n<4>();
  }
}

mf_status tc_setup(mf_operator* op, void* table_dev, cudaStream_t s) {
  if (!tc_eligible(op)) return MF_OK;
  switch (op->n) {
    case 2: tc_make_table<2>(op, op->tc_host, op->tc_fexp); break;
    case 3: tc_make_table<3>(op, op->tc_host, op->tc_fexp); break;
    default: tc_make_table<4>(op, op->tc_host, op->tc_fexp); break;
  }
  op->tc_table = table_dev;
  return cuda_check(cudaMemcpyAsync(table_dev, op->tc_host.data(), op->tc_host.size() * 2, cudaMemcpyHostToDevice, s),
                    "tensor-core table upload");
}

mf_status tc_apply(const mf_operator* op, const void* x, void* y, cudaStream_t s) {
  if (!tc_eligible(op) || !op->tc_table) return set_error(MF_ERR_UNSUPPORTED, "tensor-core apply: operator not eligible");
  switch (op->n) {
    case 2: return tc_launch_n<2>(op, x, y, s);
    case 3: return tc_launch_n<3>(op, x, y, s);
    default: return tc_launch_n<4>(op, x, y, s);
  }
}

int tc_read_error(int reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof(int)) != cudaSuccess) return -1;
  if (reset && v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_tc_error, &z, sizeof(int));
  }
  return v;
}

} // namespace mf
