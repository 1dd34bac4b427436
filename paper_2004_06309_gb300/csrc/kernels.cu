// CUDA kernels of the hz library (sm_103a).
//
//   * value assembly A(omega) = K - omega^2 M' - i omega B'        (Eq. 2)
//   * batched multifrontal complex-symmetric LDL^T of all A_i and E (the local
//     "direct solver" of the method, factorised once per frequency)
//   * batched supernodal forward / diagonal / backward solves       (Eq. 3-4)
//   * restriction R_i (gather) and PU-weighted prolongation R_i^T D_i
//   * complex CSR SpMV, real-by-complex CSR SpMV (Z, Z^T)
//   * fused CGS2 passes, deterministic reductions, Givens update    (GMRES)
//
// Complex numbers are interleaved (re, im) pairs: double2 (complex128) or
// float2 (complex64).  All reductions are fixed-order (no atomics on values),
// so reruns are bitwise identical.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "dev.h"

namespace hz {

// Kernel launches issued by this library (for the launch count in hz_stats).
static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
#define HZ_COUNT() g_launches.fetch_add(1, std::memory_order_relaxed)

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float xfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double xfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename V> struct RealOf;
template <> struct RealOf<float2> { using T = float; };
template <> struct RealOf<double2> { using T = double; };

template <typename V>
__device__ __forceinline__ V mk(typename RealOf<V>::T x, typename RealOf<V>::T y) {
  V v;
  v.x = x;
  v.y = y;
  return v;
}
template <typename V> __device__ __forceinline__ V czero() { return mk<V>(0, 0); }
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cneg(V a) { return mk<V>(-a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return mk<V>(xfma(a.x, b.x, -a.y * b.y), xfma(a.x, b.y, a.y * b.x));
}
// c + a b
template <typename V> __device__ __forceinline__ V cmad(V a, V b, V c) {
  c.x = xfma(a.x, b.x, c.x);
  c.x = xfma(-a.y, b.y, c.x);
  c.y = xfma(a.x, b.y, c.y);
  c.y = xfma(a.y, b.x, c.y);
  return c;
}
// c - a b
template <typename V> __device__ __forceinline__ V cmsub(V a, V b, V c) {
  c.x = xfma(-a.x, b.x, c.x);
  c.x = xfma(a.y, b.y, c.x);
  c.y = xfma(-a.x, b.y, c.y);
  c.y = xfma(-a.y, b.x, c.y);
  return c;
}
// c + conj(a) b
template <typename V> __device__ __forceinline__ V cmadc(V a, V b, V c) {
  c.x = xfma(a.x, b.x, c.x);
  c.x = xfma(a.y, b.y, c.x);
  c.y = xfma(a.x, b.y, c.y);
  c.y = xfma(-a.y, b.x, c.y);
  return c;
}
template <typename V> __device__ __forceinline__ V cinv(V a) {
  const typename RealOf<V>::T d = a.x * a.x + a.y * a.y;
  return mk<V>(a.x / d, -a.y / d);
}
template <typename V> __device__ __forceinline__ V from2(double2 a);
template <> __device__ __forceinline__ double2 from2<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from2<float2>(double2 a) { return make_float2(float(a.x), float(a.y)); }
__device__ __forceinline__ double2 to2(double2 a) { return a; }
__device__ __forceinline__ double2 to2(float2 a) { return make_double2(a.x, a.y); }

template <typename V> __device__ __forceinline__ V shfl_xor(V v, int m, int w = 32) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m, w);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m, w);
  return v;
}
template <typename V> __device__ __forceinline__ V warp_sum(V v) {
  for (int o = 16; o > 0; o >>= 1) v = cadd(v, shfl_xor(v, o));
  return v;
}

// widest supernode (pivot columns) any kernel handles
constexpr int kMaxK = 128;

static inline unsigned grid_for(int64_t work, int per_block, int cap = 152 * 16) {
  int64_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return unsigned(g);
}

// ---------------------------------------------------------------------------
// value assembly, Eq. (2): A = K - w^2 M' - i w B'
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 helmholtz_value(double k, double2 m, double2 b, double w) {
  // K - w^2 (m.x + i m.y) - i w (b.x + i b.y)
  return make_double2(k - w * w * m.x + w * b.y, -w * w * m.y - w * b.x);
}

__global__ void k_fill_values(int64_t nnz, const double* K, const double2* M, const double2* B, double w,
                              double2* out) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nnz; e += int64_t(gridDim.x) * blockDim.x)
    out[e] = helmholtz_value(K[e], M[e], B[e], w);
}

void launch_fill_values(int64_t nnz, const double* K, const double2* M, const double2* B, double w,
                        double2* out, cudaStream_t st) {
  if (nnz == 0) return;
  HZ_COUNT();
  k_fill_values<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, K, M, B, w, out);
}

template <typename V>
__global__ void k_front_fill(int64_t ne, const int64_t* epos, const double* K, const double2* M,
                             const double2* B, double w, V* fronts) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ne; e += int64_t(gridDim.x) * blockDim.x)
    fronts[epos[e]] = from2<V>(helmholtz_value(K[e], M[e], B[e], w));
}

// ---------------------------------------------------------------------------
// multifrontal factorisation, one assembly-tree level at a time
// ---------------------------------------------------------------------------

// Extend-add: parent front += child's contribution block (lower triangle).
// One warp per contribution column; a launch holds at most one child per parent.
template <typename V>
__global__ void __launch_bounds__(256) k_extend_add(const int2* tasks, const SnDev* sn, const int32_t* rel,
                                                    const int64_t* reloff, V* fronts) {
  const int2 t = tasks[blockIdx.x];
  const SnDev C = sn[t.x];
  const int r = C.m - C.k;
  const int b = t.y * 8 + (threadIdx.x >> 5);
  if (b >= r) return;
  const SnDev P = sn[C.parent];
  const int32_t* rl = rel + reloff[t.x];
  const V* Fc = fronts + C.frontoff;
  V* Fp = fronts + P.frontoff;
  const int64_t pc = int64_t(rl[b]) * P.m;
  const int64_t cc = int64_t(C.k + b) * C.m + C.k;
  for (int a = b + (threadIdx.x & 31); a < r; a += 32) {
    const int64_t q = pc + rl[a];
    Fp[q] = cadd(Fp[q], Fc[cc + a]);
  }
}

__device__ __forceinline__ void record_pivot(DevStatus* st, double mag, double tiny) {
  unsigned long long bits = __double_as_longlong(mag);
  atomicMin(reinterpret_cast<unsigned long long*>(&st->min_pivot), bits);
  if (!(mag >= tiny)) atomicOr(&st->zero_pivot, 1u);
}

// Pivot block: F11 = L D L^T in shared memory, then T = L^{-1} (unit lower) in
// place; the front keeps T below the diagonal and D^{-1} on it.
template <typename V>
__global__ void __launch_bounds__(256) k_diag(const int32_t* lev_sn, const SnDev* sn, V* fronts,
                                              DevStatus* status, double tiny) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* A = reinterpret_cast<V*>(smem_raw);
  const SnDev S = sn[lev_sn[blockIdx.x]];
  const int k = S.k, m = S.m, ld = k + 1;
  V* dinv = A + ld * k;
  V* row = dinv + k;
  V* F = fronts + S.frontoff;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    A[i + j * ld] = (i >= j) ? F[i + int64_t(j) * m] : czero<V>();
  }
  __syncthreads();
  for (int j = 0; j < k; j++) {
    const V d = A[j + j * ld];
    const V di = cinv(d);
    if (tid == 0) {
      dinv[j] = di;
      record_pivot(status, sqrt(double(d.x) * double(d.x) + double(d.y) * double(d.y)), tiny);
    }
    for (int c = j + 1 + wid; c < k; c += 8) {
      const V lc = cmul(A[c + j * ld], di);
      for (int i = c + lane; i < k; i += 32) A[i + c * ld] = cmsub(A[i + j * ld], lc, A[i + c * ld]);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < k; i += blockDim.x) A[i + j * ld] = cmul(A[i + j * ld], di);
    __syncthreads();
  }
  // T = L^{-1}, row by row: T[i][j] = -(L[i][j] + sum_{j<l<i} L[i][l] T[l][j])
  for (int i = 1; i < k; i++) {
    for (int l = tid; l < i; l += blockDim.x) row[l] = A[i + l * ld];
    __syncthreads();
    for (int j = tid; j < i; j += blockDim.x) {
      V acc = row[j];
      for (int l = j + 1; l < i; l++) acc = cmad(row[l], A[l + j * ld], acc);
      A[i + j * ld] = cneg(acc);
    }
    __syncthreads();
  }
  for (int e = tid; e < k * k; e += blockDim.x) {
    const int i = e % k, j = e / k;
    if (i > j) F[i + int64_t(j) * m] = A[i + j * ld];
    else if (i == j) F[i + int64_t(j) * m] = dinv[j];
  }
}

// Off-diagonal block, 32 rows per task:
//   W = F21 T^T  (= L21 D), saved to the level scratch for the Schur update,
//   G = W D^{-1} T  (= F21 F11^{-1} = L21 L11^{-1}), written over F21.
template <typename V>
__global__ void __launch_bounds__(256) k_wg(const int2* tasks, const SnDev* sn, const int64_t* scr_off,
                                            V* fronts, V* scratch) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 t = tasks[blockIdx.x];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, r = m - k;
  V* Fs = reinterpret_cast<V*>(smem_raw);  // 32 x k, ld 32
  V* Ws = Fs + 32 * k;
  V* di = Ws + 32 * k;
  V* F = fronts + S.frontoff;
  const int R0 = t.y * 32;                 // first row within the off-diagonal part
  const int nr = min(32, r - R0);
  const int tid = threadIdx.x, rr = tid & 31, g = tid >> 5;
  for (int e = tid; e < 32 * k; e += blockDim.x) {
    const int i = e & 31, j = e >> 5;
    Fs[e] = (i < nr) ? F[(k + R0 + i) + int64_t(j) * m] : czero<V>();
  }
  for (int j = tid; j < k; j += blockDim.x) di[j] = F[j + int64_t(j) * m];
  __syncthreads();
  for (int j = g; j < k; j += 8) {
    V acc = Fs[rr + 32 * j];
    for (int i = 0; i < j; i++) acc = cmad(Fs[rr + 32 * i], F[j + int64_t(i) * m], acc);
    Ws[rr + 32 * j] = acc;
  }
  __syncthreads();
  V* W = scratch + scr_off[t.x];
  for (int e = tid; e < 32 * k; e += blockDim.x) {
    const int i = e & 31, j = e >> 5;
    if (i < nr) W[(R0 + i) + int64_t(j) * r] = Ws[e];
    Fs[e] = cmul(Ws[e], di[j]);             // L21
  }
  __syncthreads();
  for (int j = g; j < k; j += 8) {
    V acc = Fs[rr + 32 * j];
    for (int i = j + 1; i < k; i++) acc = cmad(Fs[rr + 32 * i], F[i + int64_t(j) * m], acc);
    if (rr < nr) F[(k + R0 + rr) + int64_t(j) * m] = acc;
  }
}

// Schur update of the contribution block, one 32x32 lower tile per task:
//   F22[a][b] -= sum_i W[a][i] D^{-1}_i W[b][i].
template <typename V>
__global__ void __launch_bounds__(256) k_cb(const int4* tasks, const SnDev* sn, const int64_t* scr_off,
                                            V* fronts, const V* scratch) {
  __shared__ V As[16][33];
  __shared__ V Bs[16][33];
  const int4 t = tasks[blockIdx.x];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, r = m - k;
  const V* W = scratch + scr_off[t.x];
  V* F = fronts + S.frontoff;
  const int a0 = t.y * 32, b0 = t.z * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  V acc[2][2];
  for (int p = 0; p < 2; p++)
    for (int q = 0; q < 2; q++) acc[p][q] = czero<V>();
  for (int i0 = 0; i0 < k; i0 += 16) {
    for (int e = tid; e < 512; e += 256) {
      const int rr = e & 31, ii = e >> 5;
      const int i = i0 + ii;
      V av = czero<V>(), bv = czero<V>();
      if (i < k) {
        if (a0 + rr < r) av = W[(a0 + rr) + int64_t(i) * r];
        if (b0 + rr < r) bv = cmul(W[(b0 + rr) + int64_t(i) * r], F[i + int64_t(i) * m]);
      }
      As[ii][rr] = av;
      Bs[ii][rr] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 16; ii++) {
      const V x0 = As[ii][ty * 2], x1 = As[ii][ty * 2 + 1];
      const V y0 = Bs[ii][tx * 2], y1 = Bs[ii][tx * 2 + 1];
      acc[0][0] = cmad(x0, y0, acc[0][0]);
      acc[0][1] = cmad(x0, y1, acc[0][1]);
      acc[1][0] = cmad(x1, y0, acc[1][0]);
      acc[1][1] = cmad(x1, y1, acc[1][1]);
    }
    __syncthreads();
  }
  for (int p = 0; p < 2; p++)
    for (int q = 0; q < 2; q++) {
      const int a = a0 + ty * 2 + p, b = b0 + tx * 2 + q;
      if (a < r && b < r && a >= b) {
        const int64_t pos = (k + a) + int64_t(k + b) * m;
        F[pos] = csub(F[pos], acc[p][q]);
      }
    }
}

// ---------------------------------------------------------------------------
// Tensor-core (tcgen05) Schur update of complex64 fronts, one 128 x 128 lower
// tile of the contribution block per CTA (8 warps):
//   F22[a][b] -= sum_i W[a][i] d_i^{-1} W[b][i]      (complex, i < k)
// as two real products over K' = 2k, K' interleaved by complex column (2i: real parts,
// 2i + 1: imaginary parts):
//   Re = A B1^T,  Im = A B2^T,  A = (Wr, Wi),  B1 = (Br, -Bi),  B2 = (Bi, Br),  B = W diag(d^{-1}),
// each in 3xTF32 (hi*hi + hi*lo + lo*hi, hi = TF32 rounding, lo = the remainder),
// accumulated in FP32 in tensor memory (Re: columns 0-127, Im: 128-255).
// Operands are staged K-major in shared memory as 8-row x 16-byte core matrices
// (no swizzle), kTcCols complex columns (2 kTcCols K' values) per stage, in two stages
// (96 KB, two CTAs per SM): while one stage's MMAs run the 256 threads fill the other
// (thread = tile row, half of the stage's columns; every W element is read once per
// tile; a thread's loads of the next stage are issued together, right after the current
// stage's MMAs).  One elected thread issues the MMAs
// and commits each stage to that stage's mbarrier.  Every wait is bounded: a stage
// buffer is refilled only after the commit of the stage that last used it; the polls of
// these waits and of the final one are first_wait.  When one runs out the CTA raises
// status->timeout (bit 0), skips its epilogue and drains the MMAs it issued with a
// second wait of kTcDrainPolls polls on the last commit before it frees its tensor
// memory.  The MMAs read only this CTA's shared memory and write only its tensor
// memory, so they finish in bounded time and the drain ends; should it run out as well
// (a faulty tensor pipe), bit 1 is raised and the memory is still freed, because a CTA
// that exits holding tensor memory would leave later allocations on its SM waiting
// forever.  Either bit makes hz_factor return HZ_ERR_TIMEOUT and leaves the context
// unfactored.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return uint32_t(__cvta_generic_to_shared(p)); }
// Programmatic dependent launch (the triangular sweeps, one launch per tree level): a level's
// kernel lets the next level's grid start as soon as all of its CTAs are running
// (launch_dependents), and the next level reads nothing of the previous levels' results
// before griddepcontrol.wait, which returns once the previous grid has completed and its
// writes are visible.  Loads issued before the wait touch only the factor panels and the
// task descriptors, which no sweep writes.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
// 16-byte asynchronous copy global -> shared (L2 only), and the wait for all of a thread's copies
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t y;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
  return __uint_as_float(y);
}
// float offset of element (row r, k) in a 128 x 32 K-major tile of core matrices
constexpr int kTcCols = 8;                      // complex columns per stage
constexpr int kTcK = 2 * kTcCols;               // real K' values per stage
constexpr int kTcTile = 128 * kTcK;             // floats of one 128-row operand tile
__device__ __forceinline__ int tc_off(int r, int kk) {
  return ((r >> 3) * (kTcK / 4) + (kk >> 2)) * 32 + (r & 7) * 4 + (kk & 3);
}
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  // LBO = 128 B (next core matrix along K), SBO = 8 rows x kTcK x 4 B (next 8-row group),
  // version 1, no swizzle
  return uint64_t((saddr >> 4) & 0x3FFF) | (uint64_t(128 >> 4) << 16) | (uint64_t((32 * kTcK) >> 4) << 32) |
         (uint64_t(1) << 46);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t acc) {
  // D f32, A/B tf32, both K-major, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
               :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}
constexpr int kTcDrainPolls = 1 << 22;
__device__ __forceinline__ bool tc_wait(uint64_t* mbar, uint32_t phase, int polls) {
  uint32_t done = 0;
  for (int it = 0; it < polls && !done; it++)
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n" : "=r"(done) : "r"(smem_addr(mbar)), "r"(phase));
  return done != 0;
}
__device__ __forceinline__ void tc_ld32(uint32_t ta, float* out) {
  uint32_t v[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                 "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                 "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                 "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                 "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
               : "r"(ta));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 32; j++) out[j] = __uint_as_float(v[j]);
}

// Two stages of 16 complex columns (32 real K values each): Ah, Al, B1h, B1l, B2h, B2l
// per stage, 96 KB; the MMAs of one stage run while the other is refilled.
constexpr int kTcStage = 6 * kTcTile;
constexpr int kTcSmemFloats = 2 * kTcStage;     // 96 KB: two CTAs per SM
__global__ void __launch_bounds__(256) k_cb_tc(const int4* tasks, const SnDev* sn, const int64_t* scr_off,
                                               float2* fronts, const float2* scratch, DevStatus* status,
                                               int first_wait) {
  extern __shared__ __align__(1024) float tsm[];
  __shared__ float2 dinv[kMaxK];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  const int4 t = tasks[blockIdx.x];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, r = m - k, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & 127, half = tid >> 7;        // staging: tile row, and which 8 of 16 columns
  const int a0 = t.y * 128, b0 = t.z * 128;
  const float2* W = scratch + scr_off[t.x];          // r x k, column-major (ld r)
  float2* F = fronts + S.frontoff;
  for (int i = tid; i < k; i += blockDim.x) dinv[i] = F[i + int64_t(i) * m];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tmem_base)), "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(&mbar[0])), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_addr(&mbar[1])), "r"(1));
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  // K is interleaved by complex column: K' = 2i holds the real parts, 2i + 1 the imaginary
  // ones, so Re = sum A B1^T, Im = sum A B2^T with A = (Wr, Wi), B1 = (Br, -Bi), B2 = (Bi, Br)
  const int nst = (k + kTcCols - 1) / kTcCols;
  constexpr int QH = kTcCols / 2;                   // complex columns per thread per stage
  const int ra = a0 + row, rb = b0 + row;
  // a stage's 16 operand values per thread are loaded into registers in one go, the next
  // stage's right after this stage's MMAs are issued, so the loads overlap the MMAs
  float2 av[QH], bw[QH];
  auto load_stage = [&](int st) {
#pragma unroll
    for (int q = 0; q < QH; q++) {
      const int i = kTcCols * st + QH * half + q;
      av[q] = (i < k && ra < r) ? W[ra + int64_t(i) * r] : make_float2(0.f, 0.f);
      bw[q] = (i < k && rb < r) ? W[rb + int64_t(i) * r] : make_float2(0.f, 0.f);
    }
  };
  load_stage(0);
  bool ok = true;
  int issued = 0;                                    // stages whose MMAs were committed
  for (int st = 0; st < nst; st++) {
    const int b = st & 1;
    if (st >= 2) {                                   // buffer b: stage st - 2's MMAs must be done
      const bool mine = tc_wait(&mbar[b], uint32_t((st - 2) >> 1) & 1u, first_wait);
      ok = __syncthreads_and(mine) != 0;             // block-uniform
      if (!ok) break;
    }
    float* Ah = tsm + b * kTcStage;
    float* Al = Ah + kTcTile;
    float* B1h = Al + kTcTile;
    float* B1l = B1h + kTcTile;
    float* B2h = B1l + kTcTile;
    float* B2l = B2h + kTcTile;
#pragma unroll
    for (int q = 0; q < QH; q++) {
      const int i = kTcCols * st + QH * half + q;
      const float2 a = av[q];
      const float2 bv = i < k ? cmul(bw[q], dinv[i]) : make_float2(0.f, 0.f);
      const int kk = 2 * (QH * half + q);
      const int o0 = tc_off(row, kk), o1 = tc_off(row, kk + 1);
      const float arh = tf32_rna(a.x), aih = tf32_rna(a.y);
      const float brh = tf32_rna(bv.x), bih = tf32_rna(bv.y), nbih = tf32_rna(-bv.y);
      Ah[o0] = arh;
      Al[o0] = tf32_rna(a.x - arh);
      Ah[o1] = aih;
      Al[o1] = tf32_rna(a.y - aih);
      B1h[o0] = brh;
      B1l[o0] = tf32_rna(bv.x - brh);
      B1h[o1] = nbih;
      B1l[o1] = tf32_rna(-bv.y - nbih);
      B2h[o0] = bih;
      B2l[o0] = tf32_rna(bv.y - bih);
      B2h[o1] = brh;
      B2l[o1] = tf32_rna(bv.x - brh);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      for (int kk = 0; kk < kTcK / 8; kk++) {
        const uint32_t off = kk * 256;                // two core matrices (8 K values) per MMA
        const uint32_t acc0 = (st > 0 || kk > 0) ? 1u : 0u;
        const uint64_t dah = tc_desc(smem_addr(Ah) + off), dal = tc_desc(smem_addr(Al) + off);
        tc_mma(tmem, dah, tc_desc(smem_addr(B1h) + off), acc0);
        tc_mma(tmem, dah, tc_desc(smem_addr(B1l) + off), 1u);
        tc_mma(tmem, dal, tc_desc(smem_addr(B1h) + off), 1u);
        tc_mma(tmem + 128, dah, tc_desc(smem_addr(B2h) + off), acc0);
        tc_mma(tmem + 128, dah, tc_desc(smem_addr(B2l) + off), 1u);
        tc_mma(tmem + 128, dal, tc_desc(smem_addr(B2h) + off), 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                   :: "r"(smem_addr(&mbar[b])));
    }
    issued = st + 1;
    if (st + 1 < nst) load_stage(st + 1);
  }
  // the last stage's commit covers every MMA before it (they complete in order)
  const int L = issued - 1;
  uint64_t* lbar = &mbar[L & 1];
  const uint32_t lpar = uint32_t(L >> 1) & 1u;
  if (ok) {
    const bool mine = tc_wait(lbar, lpar, first_wait);
    ok = __syncthreads_and(mine) != 0;
  }
  if (!ok) {
    const bool drained = tc_wait(lbar, lpar, kTcDrainPolls);   // MMAs still in flight
    const bool all = __syncthreads_and(drained) != 0;
    if (tid == 0) atomicOr(&status->timeout, all ? 1u : 3u);
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int q4 = warp & 3, ch = warp >> 2;           // TMEM lanes 32 q4.., columns 64 ch..
    const int a = a0 + q4 * 32 + lane;
    for (int c0 = ch * 64; c0 < ch * 64 + 64; c0 += 32) {
      float re[32], im[32];
      const uint32_t ta = tmem + (uint32_t(q4 * 32) << 16) + c0;
      tc_ld32(ta, re);
      tc_ld32(ta + 128, im);
      if (a < r) {
        for (int j = 0; j < 32; j++) {
          const int bb = b0 + c0 + j;
          if (bb < r && a >= bb) {
            const int64_t pos = (k + a) + int64_t(k + bb) * m;
            float2 f = F[pos];
            f.x -= re[j];
            f.y -= im[j];
            F[pos] = f;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(256));
}

template <typename V>
__global__ void k_front_zero(const int32_t* lev_sn, const SnDev* sn, V* fronts) {
  const SnDev S = sn[lev_sn[blockIdx.x]];
  const int64_t cnt = int64_t(S.m) * S.m;
  V* f = fronts + S.frontoff;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) f[e] = czero<V>();
}

template <typename V>
__global__ void k_panel_copy(const int32_t* lev_sn, const SnDev* sn, const V* fronts, V* panels) {
  const SnDev S = sn[lev_sn[blockIdx.x]];
  const int64_t cnt = int64_t(S.ld) * S.k;
  const V* src = fronts + S.frontoff;
  V* dst = panels + S.paneloff;
  for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) {
    const int64_t j = e / S.ld, r = e % S.ld;
    dst[e] = (r < S.m) ? src[r + j * S.m] : czero<V>();    // padding rows are zero
  }
}

static size_t diag_smem(int kmax, size_t vs) { return (size_t(kmax + 1) * kmax + 2 * kmax) * vs; }
static size_t wg_smem(int kmax, size_t vs) { return (size_t(64) * kmax + kmax) * vs; }

// One tree level of one factorisation group (whole matrices whose fronts share the
// workspace at once): each task list holds, per level, the groups' tasks in order.
template <typename V>
static void factor_level_t(const FactorDev& F, int lev, int grp, double w, V* fronts, V* scratch,
                           DevStatus* status, double tiny, cudaStream_t st) {
  const int G1 = F.ngrp + 1;
  auto range = [&](const int64_t* gp, int64_t row, int64_t& b, int64_t& e) {
    b = gp[row * G1 + grp];
    e = gp[row * G1 + grp + 1];
  };
  int64_t lb, le;
  range(F.h_lev_g, lev, lb, le);
  const int64_t nb = le - lb;
  const int32_t* lsn = F.lev_sn + lb;
  if (nb > 0) {
    HZ_COUNT();
    k_front_zero<V><<<unsigned(nb), 256, 0, st>>>(lsn, F.sn, fronts);
  }
  int64_t e0, e1;
  range(F.h_ent_g, lev, e0, e1);
  if (e1 > e0) {
    HZ_COUNT();
    k_front_fill<V><<<grid_for(e1 - e0, 256), 256, 0, st>>>(e1 - e0, F.epos + e0, F.ek + e0, F.em + e0, F.eb + e0,
                                                           w, fronts);
  }
  // extend-add, one child slot per launch so that no parent entry is written twice
  for (int q = 0; q < F.max_slot; q++) {
    int64_t b, e;
    range(F.h_ea_g, int64_t(lev) * F.max_slot + q, b, e);
    if (e > b) {
      HZ_COUNT();
      k_extend_add<V><<<unsigned(e - b), 256, 0, st>>>(F.ea_tasks + b, F.sn, F.rel, F.reloff, fronts);
    }
  }
  if (nb == 0) return;
  const size_t ds = diag_smem(F.maxk, sizeof(V));
  HZ_COUNT();
  k_diag<V><<<unsigned(nb), 256, ds, st>>>(lsn, F.sn, fronts, status, tiny);
  int64_t wb, we;
  range(F.h_wg_g, lev, wb, we);
  if (we > wb) {
    HZ_COUNT();
    k_wg<V><<<unsigned(we - wb), 256, wg_smem(F.maxk, sizeof(V)), st>>>(F.wg_tasks + wb, F.sn, F.scr_off, fronts,
                                                                       scratch);
  }
  if constexpr (sizeof(V) == 8) {
    int64_t tb, te;
    range(F.h_tc_g, lev, tb, te);
    if (te > tb) {
      HZ_COUNT();
      k_cb_tc<<<unsigned(te - tb), 256, kTcSmemFloats * sizeof(float), st>>>(F.tc_tasks + tb, F.sn, F.scr_off,
                                                                            fronts, scratch, status, F.tc_wait);
    }
  } else {
    int64_t cbb, cbe;
    range(F.h_cb_g, lev, cbb, cbe);
    if (cbe > cbb) {
      HZ_COUNT();
      k_cb<V><<<unsigned(cbe - cbb), 256, 0, st>>>(F.cb_tasks + cbb, F.sn, F.scr_off, fronts, scratch);
    }
  }
  HZ_COUNT();
  k_panel_copy<V><<<unsigned(nb), 256, 0, st>>>(lsn, F.sn, fronts, (V*)F.panels);
}

static bool g_attr_done[2] = {false, false};
static void set_attrs(int prec, int kmax) {
  if (g_attr_done[prec]) return;
  const int lim = 227 * 1024;
  if (prec == 0) {
    cudaFuncSetAttribute(k_diag<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_wg<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  } else {
    cudaFuncSetAttribute(k_diag<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_cb_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemFloats * int(sizeof(float)));
    cudaFuncSetAttribute(k_wg<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  }
  g_attr_done[prec] = true;
  (void)kmax;
}

void launch_factor_level(const FactorDev& F, int lev, int grp, double w, void* fronts, void* scratch,
                         DevStatus* status, double tiny, cudaStream_t st) {
  set_attrs(F.precision, F.maxk);
  if (F.precision == 0)
    factor_level_t<double2>(F, lev, grp, w, (double2*)fronts, (double2*)scratch, status, tiny, st);
  else
    factor_level_t<float2>(F, lev, grp, w, (float2*)fronts, (float2*)scratch, status, tiny, st);
}

// ---------------------------------------------------------------------------
// batched supernodal solves  (A_i^{-1}: forward with D^{-1}, then backward)
// ---------------------------------------------------------------------------
// Loads of solve vectors (t, u, z, x) bypass L1 (ld.global.cg): each value is read
// once per sweep, so caching it in L1 only evicts panel lines.
template <typename V> __device__ __forceinline__ V ldv(const V* p);
template <> __device__ __forceinline__ float2 ldv<float2>(const float2* p) { return __ldcg(p); }
template <> __device__ __forceinline__ double2 ldv<double2>(const double2* p) { return __ldcg(p); }

template <typename V>
__global__ void k_gather(int64_t ntot, const int32_t* gidx, const double2* src, V* dst) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < ntot; q += int64_t(gridDim.x) * blockDim.x)
    dst[q] = from2<V>(src[gidx[q]]);
}

// Forward, 64 rows of one supernode per task:
//   b1 = t[pivots] + children's updates;  rows < k:  z = D^{-1} (T b1);
//   rows >= k:  u = (children's updates) - G b1.
// Forward, RT rows of one supernode per task; 256 threads = RT rows x (256 / RT)
// column groups.  64-row tasks where a tree level has many supernodes; 16-row tasks
// where it has few (the top of a single tree), so that such a level still spreads
// over every SM (its FP64 arithmetic, not its bytes, is the bound there).
template <typename V, int RT>
__device__ __forceinline__ void fwd_item(const int2 t, const SnDev* sn, const int64_t* cptr, const int64_t* cidx,
                                         const V* panels, const V* tin, V* zout, V* u) {
  constexpr int CG = 256 / RT;
  __shared__ V b1[kMaxSolveK];
  __shared__ V part[CG][RT];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, tid = threadIdx.x;
  const int64_t* cp = cptr + S.rowoff;
  const int rr = tid % RT, cg = tid / RT;
  const int r = t.y * RT + rr;
  const V* P = panels + S.paneloff;
  V acc = czero<V>(), acc2 = czero<V>();
  if constexpr (RT == 16) {
    // sparse levels: the panel values (at most kMaxK / 16 per thread) are loaded before
    // the right-hand side is gathered; the sums keep the loop's order (even q: acc)
    constexpr int MQ = kMaxK / CG;
    V pv[MQ];
    const int jmax = min(r, k);
#pragma unroll
    for (int q = 0; q < MQ; q++) {
      const int j = cg + CG * q;
      pv[q] = (r < m && j < jmax) ? P[r + int64_t(j) * S.ld] : czero<V>();
    }
    pdl_wait();
    for (int j = tid; j < k; j += blockDim.x) {
      V a = ldv(tin + S.first + j);
      for (int64_t c = cp[j]; c < cp[j + 1]; c++) a = cadd(a, ldv(u + cidx[c]));
      b1[j] = a;
    }
    __syncthreads();
    if (r < m) {
#pragma unroll
      for (int q = 0; q < MQ; q++) {
        const int j = cg + CG * q;
        if (j < jmax) {
          if (q % 2 == 0) acc = cmad(pv[q], b1[j], acc);
          else acc2 = cmad(pv[q], b1[j], acc2);
        }
      }
      // merged solve supernodes wider than kMaxK: the remaining columns, same chains
      int j = cg + CG * MQ;
      for (; j + CG < jmax; j += 2 * CG) {
        acc = cmad(P[r + int64_t(j) * S.ld], b1[j], acc);
        acc2 = cmad(P[r + int64_t(j + CG) * S.ld], b1[j + CG], acc2);
      }
      if (j < jmax) acc = cmad(P[r + int64_t(j) * S.ld], b1[j], acc);
    }
  } else {
    pdl_wait();
    for (int j = tid; j < k; j += blockDim.x) {
      V a = ldv(tin + S.first + j);
      for (int64_t c = cp[j]; c < cp[j + 1]; c++) a = cadd(a, ldv(u + cidx[c]));
      b1[j] = a;
    }
    __syncthreads();
    if (r < m) {
      const int jmax = min(r, k);
      int j = cg;
      for (; j + CG < jmax; j += 2 * CG) {
        acc = cmad(P[r + int64_t(j) * S.ld], b1[j], acc);
        acc2 = cmad(P[r + int64_t(j + CG) * S.ld], b1[j + CG], acc2);
      }
      if (j < jmax) acc = cmad(P[r + int64_t(j) * S.ld], b1[j], acc);
    }
  }
  part[cg][rr] = cadd(acc, acc2);
  __syncthreads();
  if (cg == 0 && r < m) {
    V tot = part[0][rr];
#pragma unroll
    for (int q = 1; q < CG; q++) tot = cadd(tot, part[q][rr]);
    if (r < k) {
      zout[S.first + r] = cmul(P[r + int64_t(r) * S.ld], cadd(b1[r], tot));
    } else {
      V b2 = czero<V>();
      for (int64_t c = cp[r]; c < cp[r + 1]; c++) b2 = cadd(b2, ldv(u + cidx[c]));
      u[S.uoff + (r - k)] = csub(b2, tot);
    }
  }
  __syncthreads();                                   // b1 / part are reused by the next item
}

template <typename V, int RT>
__global__ void __launch_bounds__(256) k_fwd(const int2* tasks, const SnDev* sn, const int64_t* cptr,
                                             const int64_t* cidx, const V* panels, const V* tin, V* zout,
                                             V* u) {
  pdl_trigger();
  fwd_item<V, RT>(tasks[blockIdx.x], sn, cptr, cidx, panels, tin, zout, u);
}

// Backward, split over row chunks so that tall supernodes use many CTAs:
//   partial[task][c] = sum over the task's rows r > j of P[r][j] vec[r],
//   vec = (z, -x[ancestor rows]) for 32 pivot columns j of one supernode;
// then x[j] = z[j] + sum of the partials in chunk order (deterministic).
constexpr int kBwdRows = 512;
// Fused second stage of the backward sweep ("last block done"), for a (supernode,
// column block) split over several row chunks: every partial-sum CTA of the pair
// publishes its 32 sums, fences, and bumps the pair's counter; the CTA that brings it
// to `chunks` adds the partials in chunk order (deterministic), writes x, and resets
// the counter for the next sweep.  No CTA ever waits on another.  (The single-chunk
// case finishes inside its own CTA and never touches the counter.)
template <typename V>
__device__ __forceinline__ void bwd_finish(const int4 fin, const SnDev& S, const V* zin, const V* partial_level,
                                           V* x, unsigned int* counter) {
  __shared__ unsigned int ticket;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != unsigned(fin.w) - 1) return;
  __threadfence();
  const int c = threadIdx.x;
  if (c < 32) {
    const int j = fin.y * 32 + c;
    if (j < S.k) {
      V acc = czero<V>();
      for (int ch = 0; ch < fin.w; ch++) {
        const V* pp = partial_level + int64_t(fin.z + ch) * 32 + c;
        V v;
        if constexpr (sizeof(V) == 8) {
          const float2 t = __ldcg(reinterpret_cast<const float2*>(pp));
          v.x = t.x; v.y = t.y;
        } else {
          const double2 t = __ldcg(reinterpret_cast<const double2*>(pp));
          v.x = t.x; v.y = t.y;
        }
        acc = cadd(acc, v);
      }
      x[S.first + j] = cadd(zin[S.first + j], acc);
    }
    if (c == 0) *counter = 0u;
  }
}

// complex128 backward partial sums, transposed mapping for FP64 throughput: thread
// (c, s) sums column j = 32 * block + c over slice s (of 8) of the chunk's rows,
// reading its column sequentially (L1 reuse of each 128-byte line); the 8 slice
// sums are then added in a fixed order.  No shuffle reductions on the FP64 pipe.
// PF (narrow chunks of at most 64 rows, sparse levels): each thread's <= 8 panel values are
// loaded before the chunk's right-hand side is gathered; the sums keep the loop's order.
// A supernode that fits in one chunk is finished by its own CTA, with the same sums, without
// the partial-sum round trip and ticket of bwd_finish.
template <bool PF>
__global__ void __launch_bounds__(256) k_bwd_partial_c128(const int4* tasks, const SnDev* sn,
                                                          const int32_t* rowlist, const double2* panels,
                                                          const double2* zin, double2* x, double2* partial,
                                                          int rows, const int4* fins, unsigned int* counters) {
  pdl_trigger();
  __shared__ double2 vec[kBwdRows];
  __shared__ double2 red[8][33];
  const int4 t = tasks[blockIdx.x];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, tid = threadIdx.x, c = tid & 31, s = tid >> 5;
  const int r0 = t.z * rows, r1 = min(m, r0 + rows);
  const int32_t* rl = rowlist + S.rowoff;
  const int j = t.y * 32 + c;
  const int slice = (rows + 7) / 8;
  const int ra = max(r0 + s * slice, j + 1), rb = min(r1, r0 + (s + 1) * slice);
  const double2* col = panels + S.paneloff + int64_t(j < k ? j : 0) * S.ld;
  double2 pre[8];
  if constexpr (PF) {
#pragma unroll
    for (int q = 0; q < 8; q++) {
      const int r = ra + q;
      pre[q] = (j < k && r < rb) ? col[r] : make_double2(0.0, 0.0);
    }
  }
  pdl_wait();
  for (int r = r0 + tid; r < r1; r += blockDim.x) vec[r - r0] = (r < k) ? zin[S.first + r] : cneg(x[rl[r]]);
  __syncthreads();
  double2 a0 = make_double2(0.0, 0.0), a1 = a0;
  if (j < k) {
    if constexpr (PF) {
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int r = ra + q;
        if (r < rb) {
          if (q % 2 == 0) a0 = cmad(pre[q], vec[r - r0], a0);     // the loop's pairs (r, r + 1)
          else a1 = cmad(pre[q], vec[r - r0], a1);
        }
      }
    } else {
      int r = ra;
      for (; r + 1 < rb; r += 2) {
        a0 = cmad(col[r], vec[r - r0], a0);
        a1 = cmad(col[r + 1], vec[r + 1 - r0], a1);
      }
      if (r < rb) a0 = cmad(col[r], vec[r - r0], a0);
    }
  }
  red[s][c] = cadd(a0, a1);
  __syncthreads();
  const bool single = m <= rows;                     // the only chunk: finish here, no ticket
  if (s == 0) {
    double2 tot = red[0][c];
    for (int q = 1; q < 8; q++) tot = cadd(tot, red[q][c]);
    if (!single)
      partial[int64_t(blockIdx.x) * 32 + c] = tot;
    else if (j < k)
      x[S.first + j] = cadd(zin[S.first + j], cadd(make_double2(0.0, 0.0), tot));
  }
  if (!single) bwd_finish<double2>(fins[t.w], S, zin, partial, x, counters + t.w);
}

// complex64 forward, 512 / CG rows of one supernode per task: thread t owns the row
// pair (2p, 2p+1), p = t % (256 / CG), for the pivot columns j = t / (256 / CG) mod CG,
// with 16-byte loads; the right-hand side b1 is gathered once per task.  CG = 2 (256
// rows) where a tree level has many supernodes; CG = 8 (64 rows, each warp one column
// group) on sparse levels, where a task's serial walk over its columns, not bandwidth,
// sets the time.  In both, a thread's first 8 panel values are loaded, and the update
// rows' child contributions b2 gathered, before the barrier that publishes b1, so the
// load chains overlap; with CG = 2 the next kFwdAsync values are also copied into shared
// memory (cp.async) before the gather.  Every sum keeps the order of the column loop
// (even q on one chain, odd q on the other).
constexpr int kFwdAsync = 8, kFwdNarrowAsync = 8;
template <int CG>
__device__ __forceinline__ void fwd_c64_item(const int2 t, const SnDev* sn, const int64_t* cptr,
                                             const int64_t* cidx, const float2* panels, const float2* tin,
                                             float2* zout, float2* u) {
  constexpr int NP = 256 / CG;                       // row pairs per task
  constexpr int ROWS = 2 * NP;
  __shared__ float2 b1[kMaxSolveK64];
  __shared__ float2 part[CG][ROWS];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, tid = threadIdx.x;
  const int pr = tid % NP, cg = tid / NP;
  const int64_t* cp = cptr + S.rowoff;
  const int r = t.y * ROWS + 2 * pr;                 // rows r, r + 1 (r even, ld % 4 == 0)
  const int rr = t.y * ROWS + tid;                   // update row finished by this thread
  float2 a0 = make_float2(0.f, 0.f), a1 = a0, c0 = a0, c1 = a0, b2 = a0;
  if constexpr (CG == 8) {
    constexpr int MQ = kMaxK / CG, PF = 8;              // PF of the MQ columns are prefetched,
    constexpr int NA = kFwdNarrowAsync;                 // the next NA copied by cp.async
    __shared__ __align__(16) float4 apf[NA > 0 ? NA * 256 : 1];
    float4 pv[MQ];
    const int j0 = min(r, k), j1 = min(r + 1, k);
    const float4* P4 = reinterpret_cast<const float4*>(panels + S.paneloff + (r < m ? r : 0));
    const int64_t ld4 = S.ld / 2;
#pragma unroll
    for (int q = 0; q < PF; q++) {
      const int j = cg + CG * q;
      pv[q] = (r < m && j < j1) ? P4[int64_t(j) * ld4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = PF; q < PF + NA; q++) {
      const int j = cg + CG * q;
      if (r < m && j < j1) cp_async16(&apf[(q - PF) * 256 + tid], P4 + int64_t(j) * ld4);
    }
    pdl_wait();
    for (int jj = tid; jj < k; jj += blockDim.x) {
      float2 acc = ldv(tin + S.first + jj);
      for (int64_t c = cp[jj]; c < cp[jj + 1]; c++) acc = cadd(acc, ldv(u + cidx[c]));
      b1[jj] = acc;
    }
    if (tid < ROWS && rr >= k && rr < m)
      for (int64_t c = cp[rr]; c < cp[rr + 1]; c++) b2 = cadd(b2, ldv(u + cidx[c]));
    if constexpr (NA > 0) cp_async_wait_all();        // each thread reads back only its own copies
    __syncthreads();
    if (r < m) {
#pragma unroll
      for (int q = 0; q < MQ; q++) {
        const int j = cg + CG * q;
        if (j < j1) {
          if (q >= PF && q < PF + NA) pv[q] = apf[(q - PF) * 256 + tid];
          else if (q >= PF) pv[q] = P4[int64_t(j) * ld4];
          const float2 bj = b1[j];
          if (q % 2 == 0) {
            a1 = cmad(make_float2(pv[q].z, pv[q].w), bj, a1);
            if (j < j0) a0 = cmad(make_float2(pv[q].x, pv[q].y), bj, a0);
          } else {
            c1 = cmad(make_float2(pv[q].z, pv[q].w), bj, c1);
            if (j < j0) c0 = cmad(make_float2(pv[q].x, pv[q].y), bj, c0);
          }
        }
      }
      // merged solve supernodes wider than kMaxK: the remaining columns, same chains
      int j = cg + CG * MQ;
      for (; j + CG < j1; j += 2 * CG) {
        const float4 p = P4[int64_t(j) * ld4];
        const float4 q = P4[int64_t(j + CG) * ld4];
        const float2 bj = b1[j], bq = b1[j + CG];
        a1 = cmad(make_float2(p.z, p.w), bj, a1);
        c1 = cmad(make_float2(q.z, q.w), bq, c1);
        if (j < j0) a0 = cmad(make_float2(p.x, p.y), bj, a0);
        if (j + CG < j0) c0 = cmad(make_float2(q.x, q.y), bq, c0);
      }
      if (j < j1) {
        const float4 p = P4[int64_t(j) * ld4];
        const float2 bj = b1[j];
        a1 = cmad(make_float2(p.z, p.w), bj, a1);
        if (j < j0) a0 = cmad(make_float2(p.x, p.y), bj, a0);
      }
    }
  } else {
    constexpr int PF = 8;                              // columns q < PF are prefetched
    constexpr int NA = kFwdAsync;                      // columns PF <= q < PF + NA: cp.async
    __shared__ __align__(16) float4 apf[NA > 0 ? NA * 256 : 1];
    float4 pv[PF];
    const int j0 = min(r, k), j1 = min(r + 1, k);
    const float4* P4 = reinterpret_cast<const float4*>(panels + S.paneloff + (r < m ? r : 0));
    const int64_t ld4 = S.ld / 2;
#pragma unroll
    for (int q = 0; q < PF; q++) {
      const int j = cg + CG * q;
      pv[q] = (r < m && j < j1) ? P4[int64_t(j) * ld4] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < NA; q++) {
      const int j = cg + CG * (PF + q);
      if (r < m && j < j1) cp_async16(&apf[q * 256 + tid], P4 + int64_t(j) * ld4);
    }
    pdl_wait();
    for (int jj = tid; jj < k; jj += blockDim.x) {
      float2 acc = ldv(tin + S.first + jj);
      for (int64_t c = cp[jj]; c < cp[jj + 1]; c++) acc = cadd(acc, ldv(u + cidx[c]));
      b1[jj] = acc;
    }
    if (tid < ROWS && rr >= k && rr < m)
      for (int64_t c = cp[rr]; c < cp[rr + 1]; c++) b2 = cadd(b2, ldv(u + cidx[c]));
    if constexpr (NA > 0) cp_async_wait_all();        // each thread reads back only its own copies
    __syncthreads();
    if (r < m) {
#pragma unroll
      for (int q = 0; q < PF; q++) {
        const int j = cg + CG * q;
        if (j < j1) {
          const float2 bj = b1[j];
          if (q % 2 == 0) {
            a1 = cmad(make_float2(pv[q].z, pv[q].w), bj, a1);
            if (j < j0) a0 = cmad(make_float2(pv[q].x, pv[q].y), bj, a0);
          } else {
            c1 = cmad(make_float2(pv[q].z, pv[q].w), bj, c1);
            if (j < j0) c0 = cmad(make_float2(pv[q].x, pv[q].y), bj, c0);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NA; q++) {
        const int j = cg + CG * (PF + q);
        if (j < j1) {
          const float4 p = apf[q * 256 + tid];
          const float2 bj = b1[j];
          if ((PF + q) % 2 == 0) {
            a1 = cmad(make_float2(p.z, p.w), bj, a1);
            if (j < j0) a0 = cmad(make_float2(p.x, p.y), bj, a0);
          } else {
            c1 = cmad(make_float2(p.z, p.w), bj, c1);
            if (j < j0) c0 = cmad(make_float2(p.x, p.y), bj, c0);
          }
        }
      }
      int j = cg + CG * (PF + NA);
      for (; j + CG < j1; j += 2 * CG) {               // two independent chains
        const float4 p = P4[int64_t(j) * ld4];
        const float4 q = P4[int64_t(j + CG) * ld4];
        const float2 bj = b1[j], bq = b1[j + CG];
        a1 = cmad(make_float2(p.z, p.w), bj, a1);
        c1 = cmad(make_float2(q.z, q.w), bq, c1);
        if (j < j0) a0 = cmad(make_float2(p.x, p.y), bj, a0);
        if (j + CG < j0) c0 = cmad(make_float2(q.x, q.y), bq, c0);
      }
      if (j < j1) {
        const float4 p = P4[int64_t(j) * ld4];
        const float2 bj = b1[j];
        a1 = cmad(make_float2(p.z, p.w), bj, a1);
        if (j < j0) a0 = cmad(make_float2(p.x, p.y), bj, a0);
      }
    }
  }
  part[cg][2 * pr] = cadd(a0, c0);
  part[cg][2 * pr + 1] = cadd(a1, c1);
  __syncthreads();
  if (tid < ROWS && rr < m) {
    float2 tot = part[0][tid];
#pragma unroll
    for (int q = 1; q < CG; q++) tot = cadd(tot, part[q][tid]);
    const float2* P = panels + S.paneloff;
    if (rr < k)
      zout[S.first + rr] = cmul(P[rr + int64_t(rr) * S.ld], cadd(b1[rr], tot));
    else
      u[S.uoff + (rr - k)] = csub(b2, tot);
  }
  __syncthreads();                                   // b1 / part are reused by the next item
}

template <int CG>
__global__ void __launch_bounds__(256, 4) k_fwd_c64(const int2* tasks, const SnDev* sn, const int64_t* cptr,
                                                 const int64_t* cidx, const float2* panels, const float2* tin,
                                                 float2* zout, float2* u) {
  pdl_trigger();
  fwd_c64_item<CG>(tasks[blockIdx.x], sn, cptr, cidx, panels, tin, zout, u);
}

// complex64 backward partial sums with 16-byte loads (two rows per lane), two forms:
//   kBwdAsync  (wide chunks): the first kBwdAsyncIt row pairs per lane and column are copied
//              into shared memory by asynchronous copies (cp.async, no registers held)
//              issued before the gather, so the panel stream starts while the gather's
//              dependent loads are in flight; the rest of each column is loaded in the loop;
//   kBwdPrefetch (narrow chunks of at most 128 rows, sparse levels): each lane's <= 2 row
//              pairs of its 4 columns are loaded into registers before the gather.
// Both keep the column loop's sums in its order.  The panel loads issued before the gather
// do not depend on earlier levels; the kernel waits for the previous level
// (griddepcontrol.wait, a no-op without programmatic dependent launch) only after them,
// before its first read of x.  A supernode that fits in one chunk is finished by
// its own CTA (lane 0 of each column's warp), with the same sums, without the partial-sum
// round trip and ticket of bwd_finish.
enum { kBwdAsync = 1, kBwdPrefetch = 2 };
constexpr int kBwdAsyncIt = 2;
template <int MODE>
__global__ void __launch_bounds__(256, MODE == kBwdPrefetch ? 4 : 6)
    k_bwd_partial_c64(const int4* tasks, const SnDev* sn, const int32_t* rowlist, const float2* panels,
                      const float2* zin, float2* x, float2* partial, int rows, const int4* fins,
                      unsigned int* counters) {
  pdl_trigger();
  __shared__ __align__(16) float2 vec[kBwdRows + 2];
  __shared__ __align__(16) float4 apf[MODE == kBwdAsync ? 4 * kBwdAsyncIt * 256 : 1];
  const int4 t = tasks[blockIdx.x];
  const SnDev S = sn[t.x];
  const int k = S.k, m = S.m, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int r0 = t.z * rows, r1 = min(m, r0 + rows);
  const int32_t* rl = rowlist + S.rowoff;
  float4 pre[4][2];
  if constexpr (MODE == kBwdPrefetch) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int j = t.y * 32 + wid + 8 * q;
      const float4* col = reinterpret_cast<const float4*>(panels + S.paneloff + int64_t(j < k ? j : 0) * S.ld);
      const int rs = max(r0, (j + 1) & ~1);
#pragma unroll
      for (int it = 0; it < 2; it++) {
        const int r = rs + 2 * lane + 64 * it;
        pre[q][it] = (j < k && r < r1) ? col[r >> 1] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  } else if constexpr (MODE == kBwdAsync) {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int j = t.y * 32 + wid + 8 * q;
      const float4* col = reinterpret_cast<const float4*>(panels + S.paneloff + int64_t(j < k ? j : 0) * S.ld);
      const int rs = max(r0, (j + 1) & ~1);
#pragma unroll
      for (int it = 0; it < kBwdAsyncIt; it++) {
        const int r = rs + 2 * lane + 64 * it;
        if (j < k && r < r1) cp_async16(&apf[(q * kBwdAsyncIt + it) * 256 + tid], col + (r >> 1));
      }
    }
  }
  pdl_wait();
  for (int r = r0 + tid; r < r0 + rows + 2; r += blockDim.x)
    vec[r - r0] = (r < r1) ? ((r < k) ? zin[S.first + r] : cneg(x[rl[r]])) : make_float2(0.f, 0.f);
  if constexpr (MODE == kBwdAsync) cp_async_wait_all();     // each thread reads back only its own copies
  __syncthreads();
  float2* out = partial + int64_t(blockIdx.x) * 32;
  const bool single = m <= rows;                     // the only chunk: finish here, no ticket
  const float4* vec4 = reinterpret_cast<const float4*>(vec);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int c = wid + 8 * q;
    const int j = t.y * 32 + c;
    float2 acc = make_float2(0.f, 0.f);
    if (j < k) {
      const int rs = max(r0, (j + 1) & ~1);          // first even row of the pair holding row j + 1
      if constexpr (MODE == kBwdPrefetch) {
#pragma unroll
        for (int it = 0; it < 2; it++) {
          const int r = rs + 2 * lane + 64 * it;
          if (r < r1) {
            const float4 p = pre[q][it];
            const float4 v = vec4[(r - r0) >> 1];
            if (r > j) acc = cmad(make_float2(p.x, p.y), make_float2(v.x, v.y), acc);
            acc = cmad(make_float2(p.z, p.w), make_float2(v.z, v.w), acc);
          }
        }
      } else {
        const float4* col = reinterpret_cast<const float4*>(panels + S.paneloff + int64_t(j) * S.ld);
        int r = rs + 2 * lane;
        if constexpr (MODE == kBwdAsync) {
#pragma unroll
          for (int it = 0; it < kBwdAsyncIt; it++, r += 64) {
            if (r < r1) {
              const float4 p = apf[(q * kBwdAsyncIt + it) * 256 + tid];
              const float4 v = vec4[(r - r0) >> 1];
              if (r > j) acc = cmad(make_float2(p.x, p.y), make_float2(v.x, v.y), acc);
              acc = cmad(make_float2(p.z, p.w), make_float2(v.z, v.w), acc);
            }
          }
        }
#pragma unroll 4
        for (; r < r1; r += 64) {
          const float4 p = col[r >> 1];
          const float4 v = vec4[(r - r0) >> 1];
          if (r > j) acc = cmad(make_float2(p.x, p.y), make_float2(v.x, v.y), acc);
          acc = cmad(make_float2(p.z, p.w), make_float2(v.z, v.w), acc);
        }
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      if (!single)
        out[c] = acc;
      else if (j < k)
        x[S.first + j] = cadd(zin[S.first + j], cadd(make_float2(0.f, 0.f), acc));
    }
  }
  if (!single) bwd_finish<float2>(fins[t.w], S, zin, partial, x, counters + t.w);
}

template <typename V>
__global__ void k_prolong(int64_t n, const int64_t* pptr, const int32_t* pidx, const double* pw, const V* xl,
                          const double2* y, double2* z) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n; g += int64_t(gridDim.x) * blockDim.x) {
    double2 acc = y ? y[g] : make_double2(0.0, 0.0);
    for (int64_t q = pptr[g]; q < pptr[g + 1]; q++) {
      const double2 v = to2(xl[pidx[q]]);
      acc.x = xfma(pw[q], v.x, acc.x);
      acc.y = xfma(pw[q], v.y, acc.y);
    }
    z[g] = acc;
  }
}

// One tree level of a sweep.  The complex64 sweeps launch with programmatic stream
// serialisation (unless HZ_NO_PDL is set), so that a level's CTAs start their panel loads
// while the previous level's grid drains; the kernels wait (pdl_wait) before they read any
// result of that level.  The complex128 sweeps (FP64-bound) launch plainly: on the coarse
// factor the early start measured slower (5.8 -> 6.2 ms per coarse solve on the 5 Hz
// workload).
static bool pdl_enabled(bool fp64) {
  static const bool on = std::getenv("HZ_NO_PDL") == nullptr;
  return on && !fp64;
}
template <typename... KArgs, typename... Args>
static void launch_level(void (*kern)(KArgs...), int64_t grid, cudaStream_t st, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename V>
static void solve_t(const FactorDev& F, cudaStream_t st) {
  const V* P = (const V*)F.panels;
  V* t = (V*)F.t_loc;
  V* z = (V*)F.z_loc;
  V* x = (V*)F.x_loc;
  V* u = (V*)F.u_ws;
  V* part = (V*)F.bwd_partial;
  const SnDev* SN = F.ssn ? F.ssn : F.sn;
  const bool pdl = pdl_enabled(sizeof(V) == 16);
  if (F.level_events) cudaEventRecord(F.level_events[0], st);
  for (int l = 0; l < F.snlev; l++) {
    const int64_t b = F.h_fwd_ptr[l], e = F.h_fwd_ptr[l + 1];
    if (e > b) {
      HZ_COUNT();
      const int2* tk = F.fwd_tasks + b;
      if constexpr (sizeof(V) == 8) {
        if (F.h_fwd_rt && F.h_fwd_rt[l] == 64)
          launch_level(k_fwd_c64<8>, e - b, st, pdl, tk, SN, F.cptr, F.cidx, P, t, z, u);
        else
          launch_level(k_fwd_c64<2>, e - b, st, pdl, tk, SN, F.cptr, F.cidx, P, t, z, u);
      } else if (F.h_fwd_rt && F.h_fwd_rt[l] == 16)
        launch_level(k_fwd<V, 16>, e - b, st, pdl, tk, SN, F.cptr, F.cidx, P, t, z, u);
      else
        launch_level(k_fwd<V, 64>, e - b, st, pdl, tk, SN, F.cptr, F.cidx, P, t, z, u);
    }
    if (F.level_events) cudaEventRecord(F.level_events[1 + l], st);
  }
  for (int l = F.snlev - 1; l >= 0; l--) {
    const int64_t b = F.h_bwd_ptr[l], e = F.h_bwd_ptr[l + 1];
    if (e > b) {
      HZ_COUNT();
      const int4* tk = F.bwd_tasks + b;
      const int rows = F.h_bwd_rows ? F.h_bwd_rows[l] : F.bwd_rows;
      if constexpr (sizeof(V) == 8) {
        if (rows <= 128)
          launch_level(k_bwd_partial_c64<kBwdPrefetch>, e - b, st, pdl, tk, SN, F.rowlist, P, z, x, part, rows,
                       F.bfin_tasks, F.bwd_counters);
        else
          launch_level(k_bwd_partial_c64<kBwdAsync>, e - b, st, pdl, tk, SN, F.rowlist, P, z, x, part, rows,
                       F.bfin_tasks, F.bwd_counters);
      } else {
        if (rows <= 64)
          launch_level(k_bwd_partial_c128<true>, e - b, st, pdl, tk, SN, F.rowlist, P, z, x, part, rows,
                       F.bfin_tasks, F.bwd_counters);
        else
          launch_level(k_bwd_partial_c128<false>, e - b, st, pdl, tk, SN, F.rowlist, P, z, x, part, rows,
                       F.bfin_tasks, F.bwd_counters);
      }
    }
    if (F.level_events) cudaEventRecord(F.level_events[1 + F.snlev + (F.snlev - 1 - l)], st);
  }
}

void launch_gather(const FactorDev& F, const double2* src, cudaStream_t st) {
  if (F.ntot == 0) return;
  if (F.precision == 0) {
    HZ_COUNT();
    k_gather<double2><<<grid_for(F.ntot, 256), 256, 0, st>>>(F.ntot, F.gidx, src, (double2*)F.t_loc);
  } else {
    HZ_COUNT();
    k_gather<float2><<<grid_for(F.ntot, 256), 256, 0, st>>>(F.ntot, F.gidx, src, (float2*)F.t_loc);
  }
}

void launch_solve(const FactorDev& F, cudaStream_t st) {
  if (F.precision == 0) solve_t<double2>(F, st);
  else solve_t<float2>(F, st);
}

// ---------------------------------------------------------------------------
// merged solve supernodes (complex128 and complex64 factors): a chain s_1 -> s_2 -> ... in which each
// supernode is the only child of the next and its rows below its pivots are exactly the
// next one's rows.  A supernode's panel holds T = L11^{-1} (strict lower part; D^{-1} on the
// diagonal) over G = L21 L11^{-1}.  Appending s (T_s, G_s) to the merged M (T_M, G_M, width
// w, rows P_M, P_s, R_s in that order) gives
//   T' = [[T_M, 0], [-T_s A, T_s]],  G' = [G_M(R_s) - G_s A, G_s],  A = G_M(P_s rows),
// from the block inverse of [[L11^M, 0], [L(P_s, P_M), L11^s]] (T_s taken with a unit
// diagonal in the product).  Same entries, so the sweep reads the same bytes, in fewer
// dependent levels.
// ---------------------------------------------------------------------------
// tmp (ks x w, column-major) = M[w .. w + ks, 0 .. w)
template <typename V>
__global__ void k_merge_save(const V* M, int ldm, int w, int ks, V* tmp) {
  const int64_t n = int64_t(ks) * w;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const int q = int(e % ks), c = int(e / ks);
    tmp[e] = M[(w + q) + int64_t(ldm) * c];
  }
}

// M[w + i, c] = (i >= ks ? M[w + i, c] : 0) - sum_q C(i, q) tmp[q, c] for i < ms, c < w, with
// C = [T_s (unit diagonal, upper part 0); G_s] the appended panel.  64 x 32 output tiles,
// 16-deep slices of q staged in shared memory; each thread owns 4 rows x 2 columns.  The
// sums run in the panels' precision (the complex64 factor is itself computed in FP32).
template <typename V>
__global__ void __launch_bounds__(256) k_merge_update(V* M, int ldm, int w, const V* Ps, int lds,
                                                      int ks, int ms, const V* tmp) {
  __shared__ V Cs[16][64];
  __shared__ V As[16][32];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int i0 = blockIdx.x * 64, c0 = blockIdx.y * 32;
  V acc[4][2];
#pragma unroll
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 2; b++) acc[a][b] = czero<V>();
  for (int q0 = 0; q0 < ks; q0 += 16) {
#pragma unroll
    for (int t = 0; t < 4; t++) {
      const int e = tid + 256 * t, il = e & 63, ql = e >> 6;
      const int i = i0 + il, q = q0 + ql;
      V v = czero<V>();
      if (i < ms && q < ks) {
        if (i >= ks || i > q) v = Ps[i + int64_t(lds) * q];
        else if (i == q) v = from2<V>(make_double2(1.0, 0.0));
      }
      Cs[ql][il] = v;
    }
#pragma unroll
    for (int t = 0; t < 2; t++) {
      const int e = tid + 256 * t, ql = e & 15, cl = e >> 4;
      const int q = q0 + ql, c = c0 + cl;
      As[ql][cl] = (q < ks && c < w) ? tmp[q + int64_t(ks) * c] : czero<V>();
    }
    __syncthreads();
#pragma unroll
    for (int ql = 0; ql < 16; ql++) {
      const V b0 = As[ql][2 * tx], b1 = As[ql][2 * tx + 1];
#pragma unroll
      for (int a = 0; a < 4; a++) {
        const V cv = Cs[ql][4 * ty + a];
        acc[a][0] = cmad(cv, b0, acc[a][0]);
        acc[a][1] = cmad(cv, b1, acc[a][1]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; a++) {
    const int i = i0 + 4 * ty + a;
    if (i >= ms) continue;
#pragma unroll
    for (int b = 0; b < 2; b++) {
      const int c = c0 + 2 * tx + b;
      if (c >= w) continue;
      V* o = M + (w + i) + int64_t(ldm) * c;
      *o = csub(i >= ks ? *o : czero<V>(), acc[a][b]);
    }
  }
}

// M[w + i, w + q] = Ps[i, q] for i < ms, q < ks
template <typename V>
__global__ void k_merge_put(V* M, int ldm, int w, const V* Ps, int lds, int ks, int ms) {
  const int64_t n = int64_t(ks) * ms;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(e % ms), q = int(e / ms);
    M[(w + i) + int64_t(ldm) * (w + q)] = Ps[i + int64_t(lds) * q];
  }
}

template <typename V>
static void merge_panels_t(const FactorDev& F, cudaStream_t st) {
  V* P = (V*)F.panels;
  V* tmp = (V*)F.merge_tmp;
  for (const FactorDev::MergeStep& m : F.merges) {
    V* M = P + m.moff;
    const V* Ps = P + m.soff;
    if (m.w > 0) {
      HZ_COUNT();
      k_merge_save<<<grid_for(int64_t(m.ks) * m.w, 256), 256, 0, st>>>(M, m.ldm, m.w, m.ks, tmp);
      HZ_COUNT();
      k_merge_update<<<dim3(unsigned((m.ms + 63) / 64), unsigned((m.w + 31) / 32)), 256, 0, st>>>(
          M, m.ldm, m.w, Ps, m.lds, m.ks, m.ms, tmp);
    }
    HZ_COUNT();
    k_merge_put<<<grid_for(int64_t(m.ks) * m.ms, 256), 256, 0, st>>>(M, m.ldm, m.w, Ps, m.lds, m.ks, m.ms);
  }
}

void launch_merge_panels(const FactorDev& F, cudaStream_t st) {
  if (F.merges.empty()) return;
  if (F.precision == 0) merge_panels_t<double2>(F, st);
  else merge_panels_t<float2>(F, st);
}

void launch_prolong(const FactorDev& F, const double2* y, double2* z, cudaStream_t st) {
  if (F.nglob == 0) return;
  if (F.precision == 0) {
    HZ_COUNT();
    k_prolong<double2><<<grid_for(F.nglob, 256), 256, 0, st>>>(F.nglob, F.pptr, F.pidx, F.pw,
                                                               (const double2*)F.x_loc, y, z);
  } else {
    HZ_COUNT();
    k_prolong<float2><<<grid_for(F.nglob, 256), 256, 0, st>>>(F.nglob, F.pptr, F.pidx, F.pw,
                                                              (const float2*)F.x_loc, y, z);
  }
}

// ---------------------------------------------------------------------------
// batched preconditioner for S right-hand sides (pseudo-block GMRES):
// vectors are interleaved per row, X[r * S + i].  Each factor panel element is
// read once and used for all S right-hand sides.
// ---------------------------------------------------------------------------
template <typename V, int S>
__global__ void k_gather_multi(int64_t ntot, const int32_t* gidx, const double2* src, V* dst) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < ntot * S; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t q = e / S;
    const int i = int(e % S);
    dst[e] = from2<V>(src[int64_t(gidx[q]) * S + i]);
  }
}

template <typename V, int S>
__global__ void k_prolong_multi(int64_t n, const int64_t* pptr, const int32_t* pidx, const double* pw, const V* xl,
                                const double2* y, double2* z) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * S; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t g = e / S;
    const int i = int(e % S);
    double2 acc = y ? y[e] : make_double2(0.0, 0.0);
    for (int64_t q = pptr[g]; q < pptr[g + 1]; q++) {
      const double2 v = to2(xl[int64_t(pidx[q]) * S + i]);
      acc.x = xfma(pw[q], v.x, acc.x);
      acc.y = xfma(pw[q], v.y, acc.y);
    }
    z[e] = acc;
  }
}

// Forward, 64 rows x S right-hand sides per task; 128 threads = 64 rows x 2 column parities.
template <typename V, int S>
__global__ void __launch_bounds__(128) k_fwd_multi(const int2* tasks, const SnDev* sn, const int64_t* cptr,
                                                   const int64_t* cidx, const V* panels, const V* tin, V* zout,
                                                   V* u) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* b1 = reinterpret_cast<V*>(smem_raw);               // kMaxK x S
  V* part = b1 + kMaxK * S;                               // 2 x 64 x S
  const int2 t = tasks[blockIdx.x];
  const SnDev Sn = sn[t.x];
  const int k = Sn.k, m = Sn.m, tid = threadIdx.x;
  const int64_t* cp = cptr + Sn.rowoff;
  for (int e = tid; e < k * S; e += blockDim.x) {
    const int j = e / S, i = e % S;
    V acc = tin[int64_t(Sn.first + j) * S + i];
    for (int64_t c = cp[j]; c < cp[j + 1]; c++) acc = cadd(acc, u[cidx[c] * S + i]);
    b1[e] = acc;
  }
  __syncthreads();
  const int rr = tid & 63, cg = tid >> 6;
  const int r = t.y * 64 + rr;
  V acc[S];
#pragma unroll
  for (int i = 0; i < S; i++) acc[i] = czero<V>();
  if (r < m) {
    const int jmax = min(r, k);
    const V* P = panels + Sn.paneloff + r;
    for (int j = cg; j < jmax; j += 2) {
      const V p = P[int64_t(j) * Sn.ld];
      const V* bj = b1 + j * S;
#pragma unroll
      for (int i = 0; i < S; i++) acc[i] = cmad(p, bj[i], acc[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < S; i++) part[(cg * 64 + rr) * S + i] = acc[i];
  __syncthreads();
  for (int e = tid; e < 64 * S; e += blockDim.x) {
    const int row = e / S, i = e % S;
    const int rw = t.y * 64 + row;
    if (rw >= m) continue;
    const V tot = cadd(part[row * S + i], part[(64 + row) * S + i]);
    if (rw < k) {
      zout[int64_t(Sn.first + rw) * S + i] = cmul(panels[Sn.paneloff + rw + int64_t(rw) * Sn.ld], cadd(b1[rw * S + i], tot));
    } else {
      V b2 = czero<V>();
      for (int64_t c = cp[rw]; c < cp[rw + 1]; c++) b2 = cadd(b2, u[cidx[c] * S + i]);
      u[(Sn.uoff + (rw - k)) * S + i] = csub(b2, tot);
    }
  }
}

// Backward partial sums for S right-hand sides: thread (c, slice) owns pivot column
// 32 * block + c over a quarter of the chunk's rows; slices are added in a fixed
// order; the last CTA of a (supernode, column block) finishes x (no waits).
template <typename V, int S>
__global__ void __launch_bounds__(128) k_bwd_multi(const int4* tasks, const SnDev* sn, const int32_t* rowlist,
                                                   const V* panels, const V* zin, V* x, V* partial, int rows,
                                                   const int4* fins, unsigned int* counters) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* vec = reinterpret_cast<V*>(smem_raw);              // rows x S
  V* red = vec + rows * S;                                // 4 x 32 x S
  __shared__ unsigned int ticket;
  const int4 t = tasks[blockIdx.x];
  const SnDev Sn = sn[t.x];
  const int k = Sn.k, m = Sn.m, tid = threadIdx.x, c = tid & 31, sl = tid >> 5;
  const int r0 = t.z * rows, r1 = min(m, r0 + rows);
  const int32_t* rl = rowlist + Sn.rowoff;
  for (int e = tid; e < (r1 - r0) * S; e += blockDim.x) {
    const int r = r0 + e / S, i = e % S;
    vec[e] = (r < k) ? zin[int64_t(Sn.first + r) * S + i] : cneg(x[int64_t(rl[r]) * S + i]);
  }
  __syncthreads();
  const int j = t.y * 32 + c;
  const int slice = (rows + 3) / 4;
  const int ra = max(r0 + sl * slice, j + 1), rb = min(r1, r0 + (sl + 1) * slice);
  V acc[S];
#pragma unroll
  for (int i = 0; i < S; i++) acc[i] = czero<V>();
  if (j < k) {
    const V* col = panels + Sn.paneloff + int64_t(j) * Sn.ld;
    for (int r = ra; r < rb; r++) {
      const V p = col[r];
      const V* vr = vec + (r - r0) * S;
#pragma unroll
      for (int i = 0; i < S; i++) acc[i] = cmad(p, vr[i], acc[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < S; i++) red[(sl * 32 + c) * S + i] = acc[i];
  __syncthreads();
  V* out = partial + int64_t(blockIdx.x) * 32 * S;
  for (int e = tid; e < 32 * S; e += blockDim.x) {
    V tot = red[e];
    for (int q = 1; q < 4; q++) tot = cadd(tot, red[q * 32 * S + e]);
    out[e] = tot;
  }
  // fused second stage
  const int4 fin = fins[t.w];
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(counters + t.w, 1u);
  __syncthreads();
  if (ticket != unsigned(fin.w) - 1) return;
  __threadfence();
  for (int e = tid; e < 32 * S; e += blockDim.x) {
    const int cc = e / S, i = e % S;
    const int jj = fin.y * 32 + cc;
    if (jj >= k) continue;
    V a = czero<V>();
    for (int ch = 0; ch < fin.w; ch++) {
      const V* pp = partial + (int64_t(fin.z + ch) * 32 + cc) * S + i;
      V v;
      if constexpr (sizeof(V) == 8) {
        const float2 q2 = __ldcg(reinterpret_cast<const float2*>(pp));
        v.x = q2.x; v.y = q2.y;
      } else {
        const double2 q2 = __ldcg(reinterpret_cast<const double2*>(pp));
        v.x = q2.x; v.y = q2.y;
      }
      a = cadd(a, v);
    }
    x[int64_t(Sn.first + jj) * S + i] = cadd(zin[int64_t(Sn.first + jj) * S + i], a);
  }
  if (tid == 0) counters[t.w] = 0u;
}

template <typename V, int S>
static void solve_multi_t(const FactorDev& F, const V* t_in, V* z, V* x, V* u, V* part, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    // at most 64 KB are used (S = 16, complex128); leave room for the static shared variables
    cudaFuncSetAttribute(k_fwd_multi<V, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_bwd_multi<V, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const V* P = (const V*)F.panels;
  const size_t fsm = size_t(kMaxK * S + 2 * 64 * S) * sizeof(V);
  for (int l = 0; l < F.nlev; l++) {
    const int64_t b = F.h_mfwd_ptr[l], e = F.h_mfwd_ptr[l + 1];
    if (e > b) {
      HZ_COUNT();
      k_fwd_multi<V, S><<<unsigned(e - b), 128, fsm, st>>>(F.mfwd_tasks + b, F.sn, F.cptr, F.cidx, P, t_in, z, u);
    }
  }
  const size_t bsm = size_t(F.mbwd_rows * S + 4 * 32 * S) * sizeof(V);
  for (int l = F.nlev - 1; l >= 0; l--) {
    const int64_t b = F.h_mbwd_ptr[l], e = F.h_mbwd_ptr[l + 1];
    if (e > b) {
      HZ_COUNT();
      k_bwd_multi<V, S><<<unsigned(e - b), 128, bsm, st>>>(F.mbwd_tasks + b, F.sn, F.rowlist, P, z, x, part,
                                                           F.mbwd_rows, F.mbfin_tasks, F.mbwd_counters);
    }
  }
}

template <typename V, int S>
static void prec_multi_t(const FactorDev& F, const double2* src, const double2* y, double2* dst, cudaStream_t st) {
  V* t = (V*)F.mt_loc;
  HZ_COUNT();
  k_gather_multi<V, S><<<grid_for(F.ntot * S, 256), 256, 0, st>>>(F.ntot, F.gidx, src, t);
  solve_multi_t<V, S>(F, t, (V*)F.mz_loc, (V*)F.mx_loc, (V*)F.mu_ws, (V*)F.mbwd_partial, st);
  HZ_COUNT();
  k_prolong_multi<V, S><<<grid_for(F.nglob * S, 256), 256, 0, st>>>(F.nglob, F.pptr, F.pidx, F.pw,
                                                                   (const V*)F.mx_loc, y, dst);
}

// dst = y + sum_i R_i^T D_i A_i^{-1} R_i src  (S interleaved right-hand sides)
void launch_local_multi(const FactorDev& F, int S, const double2* src, const double2* y, double2* dst,
                        cudaStream_t st) {
  if (F.precision == 0) {
    if (S == 4) prec_multi_t<double2, 4>(F, src, y, dst, st);
    else if (S == 8) prec_multi_t<double2, 8>(F, src, y, dst, st);
    else prec_multi_t<double2, 16>(F, src, y, dst, st);
  } else {
    if (S == 4) prec_multi_t<float2, 4>(F, src, y, dst, st);
    else if (S == 8) prec_multi_t<float2, 8>(F, src, y, dst, st);
    else prec_multi_t<float2, 16>(F, src, y, dst, st);
  }
}

// interleaved <-> per-right-hand-side column layouts
// Interleaving of per-slot columns: slot i reads (or writes) base + off.o[i] + r; a
// negative offset marks an empty slot, read as zero and never written.
__global__ void k_interleave(int64_t n, int S, SlotCols off, const double2* base, double2* inter) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * S; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / S;
    const int i = int(e % S);
    const int64_t o = off.o[i];
    inter[e] = (o >= 0) ? base[o + r] : make_double2(0.0, 0.0);
  }
}
__global__ void k_deinterleave(int64_t n, int S, SlotCols off, const double2* inter, double2* base) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * S; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / S;
    const int i = int(e % S);
    const int64_t o = off.o[i];
    if (o >= 0) base[o + r] = inter[e];
  }
}
void launch_interleave(int64_t n, int S, const SlotCols& off, const double2* base, double2* inter, cudaStream_t st) {
  HZ_COUNT();
  k_interleave<<<grid_for(n * S, 256), 256, 0, st>>>(n, S, off, base, inter);
}
void launch_deinterleave(int64_t n, int S, const SlotCols& off, const double2* inter, double2* base, cudaStream_t st) {
  HZ_COUNT();
  k_deinterleave<<<grid_for(n * S, 256), 256, 0, st>>>(n, S, off, inter, base);
}

// Column i of S interleaved vectors set from a plain vector (other columns untouched).
__global__ void k_interleave_put(int64_t n, int S, int i, const double2* col, double2* inter) {
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
    inter[r * S + i] = col[r];
}
void launch_interleave_put(int64_t n, int S, int i, const double2* col, double2* inter, cudaStream_t st) {
  HZ_COUNT();
  k_interleave_put<<<grid_for(n, 256), 256, 0, st>>>(n, S, i, col, inter);
}

// Point-source right-hand side written into a zeroed column: out[idx[q]] += val[q].
__global__ void k_point_rhs(PointRhs p, double2* out) {
  if (threadIdx.x == 0)
    for (int q = 0; q < p.cnt; q++) out[p.idx[q]].x += p.val[q];
}
void launch_point_rhs(const PointRhs& p, double2* out, cudaStream_t st) {
  HZ_COUNT();
  k_point_rhs<<<1, 32, 0, st>>>(p, out);
}

// Y = A X (or SUB - A X) for S interleaved vectors; lanes of a warp split the right-hand sides.
template <int S>
__global__ void __launch_bounds__(256) k_spmv_multi(int64_t n, const int64_t* rp, const int32_t* ci,
                                                    const double2* val, const double2* x, const double2* sub,
                                                    double2* y) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * S; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = e / S;
    const int i = int(e % S);
    double2 a0 = make_double2(0.0, 0.0), a1 = a0;
    const int64_t q1 = rp[row + 1];
    int64_t q = rp[row];
    for (; q + 1 < q1; q += 2) {
      a0 = cmad(val[q], x[int64_t(ci[q]) * S + i], a0);
      a1 = cmad(val[q + 1], x[int64_t(ci[q + 1]) * S + i], a1);
    }
    if (q < q1) a0 = cmad(val[q], x[int64_t(ci[q]) * S + i], a0);
    const double2 acc = cadd(a0, a1);
    y[e] = sub ? csub(sub[e], acc) : acc;
  }
}
template <int S>
__global__ void __launch_bounds__(256) k_spmv_real_multi(int64_t n, const int64_t* rp, const int32_t* ci,
                                                         const double* val, const double2* x, double2* y) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n * S; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t row = e / S;
    const int i = int(e % S);
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t q = rp[row]; q < rp[row + 1]; q++) {
      const double2 v = x[int64_t(ci[q]) * S + i];
      acc.x = xfma(val[q], v.x, acc.x);
      acc.y = xfma(val[q], v.y, acc.y);
    }
    y[e] = acc;
  }
}
void launch_spmv_multi(int64_t n, int S, const int64_t* rp, const int32_t* ci, const double2* val, const double2* x,
                       const double2* sub, double2* y, cudaStream_t st) {
  HZ_COUNT();
  const unsigned g = grid_for(n * S, 256, 152 * 32);
  if (S == 4) k_spmv_multi<4><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
  else if (S == 8) k_spmv_multi<8><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
  else k_spmv_multi<16><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
}
void launch_spmv_real_multi(int64_t n, int S, const int64_t* rp, const int32_t* ci, const double* val,
                            const double2* x, double2* y, cudaStream_t st) {
  HZ_COUNT();
  const unsigned g = grid_for(n * S, 256, 152 * 32);
  if (S == 4) k_spmv_real_multi<4><<<g, 256, 0, st>>>(n, rp, ci, val, x, y);
  else if (S == 8) k_spmv_real_multi<8><<<g, 256, 0, st>>>(n, rp, ci, val, x, y);
  else k_spmv_real_multi<16><<<g, 256, 0, st>>>(n, rp, ci, val, x, y);
}

// ---------------------------------------------------------------------------
// sparse matrix-vector products
// ---------------------------------------------------------------------------
template <int TPR>
__global__ void __launch_bounds__(256) k_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double2* val,
                                              const double2* x, const double2* sub, double2* y) {
  const int lane = threadIdx.x % TPR;
  const int64_t groups = (int64_t(gridDim.x) * blockDim.x) / TPR;
  const int64_t g0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / TPR;
  const int64_t wbase0 = (blockIdx.x * int64_t(blockDim.x) + (threadIdx.x & ~31)) / TPR;
  for (int64_t off = 0; wbase0 + off < n; off += groups) {
    const int64_t row = g0 + off;
    double2 acc = make_double2(0.0, 0.0);
    if (row < n) {
      const int64_t e = rp[row + 1];
      for (int64_t q = rp[row] + lane; q < e; q += TPR) acc = cmad(val[q], x[ci[q]], acc);
    }
    for (int o = TPR / 2; o > 0; o >>= 1) acc = cadd(acc, shfl_xor(acc, o, TPR));
    if (row < n && lane == 0) y[row] = sub ? csub(sub[row], acc) : acc;
  }
}

__global__ void __launch_bounds__(256) k_spmv_real(int64_t n, const int64_t* rp, const int32_t* ci,
                                                   const double* val, const double2* x, double2* y) {
  constexpr int TPR = 4;
  const int lane = threadIdx.x % TPR;
  const int64_t groups = (int64_t(gridDim.x) * blockDim.x) / TPR;
  const int64_t g0 = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) / TPR;
  const int64_t wbase0 = (blockIdx.x * int64_t(blockDim.x) + (threadIdx.x & ~31)) / TPR;
  for (int64_t off = 0; wbase0 + off < n; off += groups) {
    const int64_t row = g0 + off;
    double2 acc = make_double2(0.0, 0.0);
    if (row < n) {
      const int64_t e = rp[row + 1];
      for (int64_t q = rp[row] + lane; q < e; q += TPR) {
        const double2 v = x[ci[q]];
        acc.x = xfma(val[q], v.x, acc.x);
        acc.y = xfma(val[q], v.y, acc.y);
      }
    }
    for (int o = TPR / 2; o > 0; o >>= 1) acc = cadd(acc, shfl_xor(acc, o, TPR));
    if (row < n && lane == 0) y[row] = acc;
  }
}

// Lanes per row for the complex SpMV (set per context by its autotuner).
static thread_local int g_spmv_tpr = 8;
void set_spmv_lanes(int tpr) { g_spmv_tpr = tpr; }

void launch_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double2* val, const double2* x,
                 const double2* sub, double2* y, cudaStream_t st) {
  if (n == 0) return;
  HZ_COUNT();
  const int t = g_spmv_tpr;
  const unsigned g = grid_for(n * t, 256, 152 * 32);
  if (t == 2) k_spmv<2><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
  else if (t == 4) k_spmv<4><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
  else if (t == 16) k_spmv<16><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
  else k_spmv<8><<<g, 256, 0, st>>>(n, rp, ci, val, x, sub, y);
}

void launch_spmv_real(int64_t n, const int64_t* rp, const int32_t* ci, const double* val, const double2* x,
                      double2* y, cudaStream_t st) {
  if (n == 0) return;
  HZ_COUNT();
  k_spmv_real<<<grid_for(n * 4, 256, 152 * 32), 256, 0, st>>>(n, rp, ci, val, x, y);
}

// ---------------------------------------------------------------------------
// GMRES: fused CGS passes and small dense updates
// ---------------------------------------------------------------------------
constexpr int kMaxCols = 64;
constexpr int kPartStride = kMaxCols + 1;
int cgs_blocks() { return 152 * 4; }

// Multi-dot: partial[b][j] = sum over the block's rows of conj(V[r][j]) w[r] (j < ncols);
// partial[b][64] = sum |w[r]|^2.  One warp per column, lanes over rows.
__device__ __forceinline__ void mdot_block(int64_t n, int ncols, const double2* __restrict__ V, int64_t ldv,
                                           const double2* __restrict__ w, double2* out, int64_t chunk, int bx) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = bx * chunk;
  const int64_t row1 = min(n, row0 + chunk);
  for (int j = wid; j < kMaxCols; j += 8) {
    double2 acc = make_double2(0.0, 0.0);
    if (j < ncols) {
      const double2* col = V + int64_t(j) * ldv;
#pragma unroll 4
      for (int64_t r = row0 + lane; r < row1; r += 32) acc = cmadc(col[r], w[r], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[j] = acc;
  }
  if (wid == 0) {
    double s = 0.0;
    for (int64_t r = row0 + lane; r < row1; r += 32) {
      const double2 v = w[r];
      s = xfma(v.x, v.x, xfma(v.y, v.y, s));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[kMaxCols] = make_double2(s, 0.0);
  }
}
__global__ void __launch_bounds__(256) k_mdot(int64_t n, int ncols, const double2* __restrict__ V, int64_t ldv,
                                              const double2* __restrict__ w, double2* partial, int64_t chunk) {
  mdot_block(n, ncols, V, ldv, w, partial + int64_t(blockIdx.x) * kPartStride, chunk, blockIdx.x);
}

// Multi-axpy: w[r] -= sum_j V[r][j] h[j]; partial[b][64] = sum |w[r]|^2 (new w).
__device__ __forceinline__ void maxpy_block(int64_t n, int ncols, const double2* __restrict__ V, int64_t ldv,
                                            const double2* __restrict__ h, double2* w, double2* out, int64_t chunk,
                                            int bx) {
  __shared__ double2 hs[kMaxCols];
  __shared__ double red[8];
  for (int j = threadIdx.x; j < ncols; j += blockDim.x) hs[j] = h[j];
  __syncthreads();
  const int64_t row0 = bx * chunk;
  const int64_t row1 = min(n, row0 + chunk);
  double s = 0.0;
  for (int64_t r = row0 + threadIdx.x; r < row1; r += blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
#pragma unroll 4
    for (int j = 0; j < ncols; j++) acc = cmad(V[r + int64_t(j) * ldv], hs[j], acc);
    const double2 v = csub(w[r], acc);
    w[r] = v;
    s = xfma(v.x, v.x, xfma(v.y, v.y, s));
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; q++) t += red[q];
    out[kMaxCols] = make_double2(t, 0.0);
  }
}
__global__ void __launch_bounds__(256) k_maxpy(int64_t n, int ncols, const double2* __restrict__ V, int64_t ldv,
                                               const double2* __restrict__ h, double2* w, double2* partial,
                                               int64_t chunk) {
  maxpy_block(n, ncols, V, ldv, h, w, partial + int64_t(blockIdx.x) * kPartStride, chunk, blockIdx.x);
}

static int64_t cgs_chunk(int64_t n) {
  const int nb = cgs_blocks();
  int64_t chunk = (n + nb - 1) / nb;
  return (chunk + 31) / 32 * 32;
}

// ndot > 0 and h == null: dots of w with V (and |w|^2); h != null: w -= V h (and |w|^2),
// followed by the dots of the updated w when ndot > 0.
void launch_cgs(int64_t n, int ncols, const double2* V, int64_t ldv, const double2* h, double2* w, int ndot,
                double2* partial, cudaStream_t st) {
  const int nb = cgs_blocks();
  const int64_t chunk = cgs_chunk(n);
  if (h) {
    HZ_COUNT();
    k_maxpy<<<nb, 256, 0, st>>>(n, ncols, V, ldv, h, w, partial, chunk);
  }
  if (ndot > 0 || !h) {
    HZ_COUNT();
    k_mdot<<<nb, 256, 0, st>>>(n, ndot, V, ldv, w, partial, chunk);
  }
}

// out[j] = sum over blocks of partial[b][j]; one CTA per j, fixed-order tree.
__device__ __forceinline__ void reduce_block(const double2* partial, int nblk, double2* out, int j) {
  __shared__ double2 red[256];
  double2 s = make_double2(0.0, 0.0);
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s = cadd(s, partial[int64_t(b) * kPartStride + j]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = cadd(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = red[0];
}
__global__ void __launch_bounds__(256) k_reduce(const double2* partial, int nblk, double2* out) {
  reduce_block(partial, nblk, out, blockIdx.x);
}

// Sums all 65 slots (columns and the norm slot 64).
void launch_reduce(const double2* partial, int nblk, int ncols, double2* out, cudaStream_t st) {
  (void)ncols;
  HZ_COUNT();
  k_reduce<<<kMaxCols + 1, 256, 0, st>>>(partial, nblk, out);
}

// Complex Givens rotation zeroing b: rho = sqrt(|a|^2+|b|^2), c = |a|/rho,
// s = (a/|a|) conj(b)/rho; a = 0 gives c = 0, s = 1.
__device__ void givens_cs(double2 a, double2 b, double& c, double2& s) {
  const double aa = sqrt(a.x * a.x + a.y * a.y);
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    return;
  }
  const double bb = sqrt(b.x * b.x + b.y * b.y);
  const double rho = sqrt(aa * aa + bb * bb);
  c = aa / rho;
  const double2 u = make_double2(a.x / aa, a.y / aa);
  const double2 bc = make_double2(b.x / rho, -b.y / rho);
  s = cmul(u, bc);
}

// Givens update of column j of the Hessenberg matrix.  The CGS coefficients of the
// Arnoldi basis start at h1/h2[off] (the first `off` are those of a recycled space,
// GCRO-DR); raw_h / raw_b (optional) keep the unrotated column and those `off`
// coefficients for the cycle-end harmonic Ritz problem.
__device__ void k_givens_body(int j, int m, double2* H, double* cs, double2* sn, double2* g, const double2* h1,
                              const double2* h2, const double2* nrm, const double* bnorm_p, double* est,
                              int* breakdown, double* invh, int off = 0, double2* raw_h = nullptr,
                              double2* raw_b = nullptr, int ldb = 0) {
  if (threadIdx.x != 0) return;
  const double bnorm = *bnorm_p;
  double2* col = H + int64_t(j) * (m + 1);
  for (int i = 0; i <= j; i++) col[i] = cadd(h1[off + i], h2[off + i]);
  const double w0 = sqrt(h1[kMaxCols].x);
  const double hn = sqrt(nrm[kMaxCols].x);
  col[j + 1] = make_double2(hn, 0.0);
  if (raw_h) {
    for (int i = 0; i <= j + 1; i++) raw_h[int64_t(j) * (m + 1) + i] = col[i];
    for (int i = 0; i < off; i++) raw_b[int64_t(j) * ldb + i] = cadd(h1[i], h2[i]);
  }
  for (int i = 0; i < j; i++) {
    const double2 a = col[i], b = col[i + 1];
    const double2 sc = make_double2(sn[i].x, -sn[i].y);
    col[i] = cadd(make_double2(cs[i] * a.x, cs[i] * a.y), cmul(sn[i], b));
    col[i + 1] = csub(make_double2(cs[i] * b.x, cs[i] * b.y), cmul(sc, a));
  }
  double c;
  double2 s;
  givens_cs(col[j], col[j + 1], c, s);
  cs[j] = c;
  sn[j] = s;
  col[j] = cadd(make_double2(c * col[j].x, c * col[j].y), cmul(s, col[j + 1]));
  col[j + 1] = make_double2(0.0, 0.0);
  const double2 gj = g[j];
  const double2 sc = make_double2(-s.x, s.y);   // -conj(s)
  g[j + 1] = cmul(sc, gj);
  g[j] = make_double2(c * gj.x, c * gj.y);
  *est = sqrt(g[j + 1].x * g[j + 1].x + g[j + 1].y * g[j + 1].y) / bnorm;
  *breakdown = (hn <= 1e-14 * w0) ? 1 : 0;
  *invh = 1.0 / hn;
}
__global__ void k_givens(int j, int m, double2* H, double* cs, double2* sn, double2* g, const double2* h1,
                         const double2* h2, const double2* nrm, const double* bnorm_p, double* est,
                         int* breakdown, double* invh, int off, double2* raw_h, double2* raw_b, int ldb) {
  if (blockIdx.x != 0) return;
  k_givens_body(j, m, H, cs, sn, g, h1, h2, nrm, bnorm_p, est, breakdown, invh, off, raw_h, raw_b, ldb);
}

void launch_givens(int j, int m, double2* H, double* cs, double2* sn, double2* g, const double2* h1,
                   const double2* h2, const double2* nrm, const double* bnorm, double* est, int* breakdown,
                   double* invh, cudaStream_t st, int off, double2* raw_h, double2* raw_b, int ldb) {
  HZ_COUNT();
  k_givens<<<1, 32, 0, st>>>(j, m, H, cs, sn, g, h1, h2, nrm, bnorm, est, breakdown, invh, off, raw_h, raw_b, ldb);
}

// ---------------------------------------------------------------------------
// The same CGS2 / Givens / scaling steps for the S slots of a pseudo-block solve in one
// launch each (grid.y = slot); each slot's arithmetic is the single-vector kernels'
// block for block, so its results do not depend on the other slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_cgs_slots(int64_t n, SlotCgs p, double2* partial, int64_t chunk,
                                                   int mode) {
  const int i = blockIdx.y, nb = gridDim.x;
  if (p.ncols[i] < 0) return;
  double2* out = partial + (int64_t(i) * nb + blockIdx.x) * kPartStride;
  if (mode == 0)
    mdot_block(n, p.ncols[i], p.V[i], n, p.w[i], out, chunk, blockIdx.x);
  else
    maxpy_block(n, p.ncols[i], p.V[i], n, p.h[i], p.w[i], out, chunk, blockIdx.x);
}
__global__ void __launch_bounds__(256) k_reduce_slots(const double2* partial, int nblk, SlotCgs p, double2* out) {
  const int i = blockIdx.y;
  if (p.ncols[i] < 0) return;
  reduce_block(partial + int64_t(i) * nblk * kPartStride, nblk, out + int64_t(i) * kPartStride, blockIdx.x);
}
void launch_cgs_slots(int64_t n, int S, const SlotCgs& p, bool maxpy, bool dots, double2* partial, double2* out,
                      cudaStream_t st) {
  const int nb = cgs_blocks();
  const int64_t chunk = cgs_chunk(n);
  if (maxpy) {
    HZ_COUNT();
    k_cgs_slots<<<dim3(nb, S), 256, 0, st>>>(n, p, partial, chunk, 1);
  }
  if (dots) {
    HZ_COUNT();
    k_cgs_slots<<<dim3(nb, S), 256, 0, st>>>(n, p, partial, chunk, 0);
  }
  HZ_COUNT();
  k_reduce_slots<<<dim3(kMaxCols + 1, S), 256, 0, st>>>(partial, nb, p, out);
}
__global__ void k_givens_slots(SlotGivens p) {
  const int i = blockIdx.x;
  if (p.j[i] < 0) return;
  const int m = p.m;
  k_givens_body(p.j[i], m, p.H + int64_t(i) * (m + 1) * m, p.cs + int64_t(i) * m, p.sn + int64_t(i) * m,
                p.g + int64_t(i) * (m + 1), p.h1 + int64_t(i) * kPartStride, p.h2 + int64_t(i) * kPartStride,
                p.nrm + int64_t(i) * kPartStride, p.scal + int64_t(i) * 8 + 4, p.scal + int64_t(i) * 8,
                p.brk + i, p.scal + int64_t(i) * 8 + 1);
}
void launch_givens_slots(int S, const SlotGivens& p, cudaStream_t st) {
  HZ_COUNT();
  k_givens_slots<<<S, 32, 0, st>>>(p);
}
__global__ void k_scale_slots(int64_t n, SlotScale p) {
  const int i = blockIdx.y;
  if (!p.out[i]) return;
  const double a = *p.s[i];
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
    p.out[i][r] = make_double2(p.w[i][r].x * a, p.w[i][r].y * a);
}
void launch_scale_slots(int64_t n, int S, const SlotScale& p, cudaStream_t st) {
  HZ_COUNT();
  k_scale_slots<<<dim3(std::max(1u, grid_for(n, 256) / unsigned(S)), S), 256, 0, st>>>(n, p);
}

// out[:, q] (+)= sign * (sum_i B1[:, i] coef[i, q] + sum_i B2[:, i] coef[nb1 + i, q]), q < nout:
// linear combinations of two column-major bases (recycled-space updates of GCRO-DR).
// coef is (nb1 + nb2) x nout column-major, staged in shared memory.
constexpr int kComboCols = 80, kComboOut = 16;
__global__ void __launch_bounds__(256) k_combo(int64_t n, int nb1, const double2* B1, int64_t ld1, int nb2,
                                               const double2* B2, int64_t ld2, const double2* coef, int nout,
                                               double2* out, int64_t ldo, double sign, int accumulate) {
  __shared__ double2 cf[kComboCols * kComboOut];
  const int nbt = nb1 + nb2;
  for (int e = threadIdx.x; e < nbt * nout; e += blockDim.x) cf[e] = coef[e];
  __syncthreads();
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    double2 acc[kComboOut];
#pragma unroll
    for (int q = 0; q < kComboOut; q++) acc[q] = make_double2(0.0, 0.0);
    for (int i = 0; i < nbt; i++) {
      const double2 v = i < nb1 ? B1[r + int64_t(i) * ld1] : B2[r + int64_t(i - nb1) * ld2];
#pragma unroll
      for (int q = 0; q < kComboOut; q++)
        if (q < nout) acc[q] = cmad(v, cf[q * nbt + i], acc[q]);
    }
    for (int q = 0; q < nout; q++) {
      double2* o = out + r + int64_t(q) * ldo;
      const double2 a = make_double2(sign * acc[q].x, sign * acc[q].y);
      *o = accumulate ? cadd(*o, a) : a;
    }
  }
}
void launch_combo(int64_t n, int nb1, const double2* B1, int64_t ld1, int nb2, const double2* B2, int64_t ld2,
                  const double2* coef, int nout, double2* out, int64_t ldo, double sign, bool accumulate,
                  cudaStream_t st) {
  if (n == 0 || nout == 0) return;
  HZ_COUNT();
  k_combo<<<grid_for(n, 256), 256, 0, st>>>(n, nb1, B1, ld1, nb2, B2, ld2, coef, nout, out, ldo, sign,
                                            accumulate ? 1 : 0);
}

__global__ void k_init_cycle(const double2* nrm2, double2* g, int m, double* invbeta, double* beta) {
  const double b = sqrt(nrm2[kMaxCols].x);
  for (int i = threadIdx.x; i <= m; i += blockDim.x) g[i] = make_double2(i == 0 ? b : 0.0, 0.0);
  if (threadIdx.x == 0) {
    *beta = b;
    *invbeta = 1.0 / b;
  }
}

void launch_init_cycle(const double2* nrm2, double2* g, int m, double* invbeta, double* beta, cudaStream_t st) {
  HZ_COUNT();
  k_init_cycle<<<1, 64, 0, st>>>(nrm2, g, m, invbeta, beta);
}

__global__ void k_scale(int64_t n, const double2* w, const double* s, double2* out) {
  const double a = *s;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = make_double2(w[i].x * a, w[i].y * a);
}

void launch_scale(int64_t n, const double2* w, const double* s, double2* out, cudaStream_t st) {
  HZ_COUNT();
  k_scale<<<grid_for(n, 256), 256, 0, st>>>(n, w, s, out);
}

// y = R^{-1} g (upper triangular k x k of the rotated Hessenberg matrix)
__global__ void k_backsub(int k, const double2* H, int ldh, const double2* g, double2* y) {
  if (threadIdx.x != 0) return;
  for (int i = k - 1; i >= 0; i--) {
    double2 s = g[i];
    for (int l = i + 1; l < k; l++) s = cmsub(H[i + int64_t(l) * ldh], y[l], s);
    const double2 d = H[i + int64_t(i) * ldh];
    y[i] = cmul(s, cinv(d));
  }
}

__global__ void k_gemv_add(int64_t n, int k, const double2* y, const double2* Zs, int64_t ldz, double2* x) {
  __shared__ double2 ys[kMaxCols];
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x) {
    double2 acc = x[r];
    for (int j = 0; j < k; j++) acc = cmad(Zs[r + int64_t(j) * ldz], ys[j], acc);
    x[r] = acc;
  }
}

// x += Zs[:, 0:k) y (k <= 64)
void launch_gemv_add(int64_t n, int k, const double2* y, const double2* Zs, int64_t ldz, double2* x, cudaStream_t st) {
  HZ_COUNT();
  k_gemv_add<<<grid_for(n, 256), 256, 0, st>>>(n, k, y, Zs, ldz, x);
}

void launch_update_x(int64_t n, int k, const double2* H, int ldh, const double2* g, double2* y, const double2* Zs,
                     int64_t ldz, double2* x, cudaStream_t st) {
  HZ_COUNT();
  k_backsub<<<1, 32, 0, st>>>(k, H, ldh, g, y);
  HZ_COUNT();
  k_gemv_add<<<grid_for(n, 256), 256, 0, st>>>(n, k, y, Zs, ldz, x);
}

__global__ void k_add2(int n, const double2* a, const double2* b, double2* out) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = cadd(a[i], b[i]);
}

void launch_add2(int n, const double2* a, const double2* b, double2* out, cudaStream_t st) {
  HZ_COUNT();
  k_add2<<<1, 64, 0, st>>>(n, a, b, out);
}

__global__ void k_copy(int64_t n, const double2* a, double2* out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    out[i] = a[i];
}

void launch_axpby_copy(int64_t n, const double2* a, double2* out, cudaStream_t st) {
  HZ_COUNT();
  k_copy<<<grid_for(n, 256), 256, 0, st>>>(n, a, out);
}

}  // namespace hz
