// lbm_mix.cu — sm_103a implementation of the C ABI in include/lbm_mix.h.
//
// One time step of the two-species D2Q9 MRT lattice Boltzmann model of
// Wang, Xu & Guo (arXiv:1603.08221, Sec. 3) is ONE fused kernel launch
// (lbm_step_kernel; on grids of two or more waves and with 16-bit storage,
// lbm_walls_kernel computes the wall parameters r and tau_q of every column
// ahead of it): pull-streaming from the previous post-collision buffer
// with the diffuse-bounce-back walls (Eqs. bot, bot2, R) and the
// extrapolation-correction ends (Eqs. rho1, rho2) folded into the loads,
// moments (Eq. rhou), effective relaxation times (Eqs. EQFrb, EQFrsp, psi,
// taos, taoq, A12), the MRT collision (Eqs. MR, m, S, feq) for both species,
// the store of the new post-collision buffer, and FP64 per-column reductions
// that feed the next step's density correction and the separation
// diagnostics (Eqs. C, CL, Clline).
//
// Data layout in HBM (per buffer): the channel is cut into strips of 32
// columns; strip s holds, row after row, the nine populations of its 32
// columns, each as one segment of 32 species pairs (a, b):
//   offset(sp, i, j, x) = (x / 32) * SS + j * RS + i * 64 + 2 * (x % 32) + sp
// with RS = 576 elements per strip row and SS = N * RS per strip.  A node's
// two species of population i are adjacent, so one 8-byte (FP32) or 4-byte
// (BF16/FP16) access per lane fetches both and a warp access is one aligned
// contiguous segment; all offsets inside a strip are compile-time
// immediates.  Two buffers A/B alternate.  The CTAs of one strip (one per
// row block) sweep their rows in steps of TY; the per-column quantities (the
// tau_q of the two walls, the column sums) are produced by the CTAs of that
// strip alone, without floating-point atomics and in a fixed order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <time.h>
#include <string.h>

#include <mutex>
#include <new>

#include "../../include/lbm_mix.h"

namespace {

// ---------------------------------------------------------------- errors
thread_local char g_err[512] = "";

int set_err(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int set_err(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                      \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return set_err(LBM_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                     __FILE__, __LINE__);                                             \
  } while (0)

// ------------------------------------------------------- lattice constants
constexpr int TX = 32;          // columns per CTA = strip width (one warp per row segment)
constexpr int RS = 18 * TX;     // elements per row of a strip (9 populations x 32 pairs)
constexpr int PS = 2 * TX;      // elements per population segment (32 columns x 2 species)
constexpr int TY = 8;           // rows per sweep iteration
constexpr int NPART = 8;        // doubles per CTA partial
constexpr int NREC = 8;         // doubles per diagnostic record
constexpr int DIAG_CAP = 4096;  // diagnostic records kept
constexpr float kPi = 3.14159265358979323846f;

struct Lat {
  int N, Nx, pitch;
  unsigned SS;           // floats per strip: N * RS
  int x_periodic;
  int wall_mode;         // LBM_WALL_DBB or LBM_WALL_BSR
  int r_form;            // LBM_R_FIRST, LBM_R_SPECIES or LBM_R_SECOND (Eq. R)
  int lam_mix;           // lambda_s with the mixture (1) or partial (0) pressure
  float rsqrt_mh[2];     // 1 / sqrt(m_s / m_min)
  int light;             // index of the light species
  float s[2];            // s_sigma = m_min / m_sigma
  float cw0[2];          // rest-equilibrium weights w_i alpha_si: rest (9 - 5s)/9,
  float cw1[2], cw5[2];  // axis s/9, diagonal s/36
  // coefficients of the non-equilibrium energy moments on the deviations
  // (rest, axis, diagonal): e: -2s, 3 - 2s, 6 - 2s; eps: 3s, 3s - 6, 3s - 3
  float ke[2][3], kp[2][3];
  // the same per-species constants as (species a, species b) pairs for the
  // packed FP32x2 arithmetic
  float2 s2, cw1_2, cw5_2, c_xl2, inv_c_xl2, ke2[3], kp2[3];
  float inv_c_lam;       // 1 / (3 mu sqrt(pi/6))
  float c_lam;           // 3 mu sqrt(pi/6): lambda = c_lam / (n sqrt(m_x))
  float c_xl[2];         // 3 mu_s sqrt(pi/(6 m_s)): x_s lambda_s = c_xl / n
  float inv_c_xl[2];
  float c_ts;            // sqrt(6/pi)
  float c_td;            // (3/2) sqrt(3 m0 m_a m_b / m_min)
  float om_e, om_eps;    // 1/tau_e, 1/tau_eps
  float c_m0;
  float H;               // channel height = N
  double mh[2];          // m_sigma / m_min
  double rho_in[2], rho_out[2];
  double C_in, C_out;    // light-species mole fraction at the ends
};

// ------------------------------------------------------ special functions
// E_1(x) for 0 < x <= 1 from its convergent series (Abramowitz & Stegun
// 5.1.11) truncated after ten terms (remainder < 2.3e-9 at x = 1):
// E_1(x) = -gamma - ln x + sum_{k=1}^{10} (-1)^{k+1} x^k / (k k!).
__device__ __forceinline__ float e1_series(float x) {
  float p = -1.0f / 36288000.0f;
  p = fmaf(p, x, 1.0f / 3265920.0f);
  p = fmaf(p, x, -1.0f / 322560.0f);
  p = fmaf(p, x, 1.0f / 35280.0f);
  p = fmaf(p, x, -1.0f / 4320.0f);
  p = fmaf(p, x, 1.0f / 600.0f);
  p = fmaf(p, x, -1.0f / 96.0f);
  p = fmaf(p, x, 1.0f / 18.0f);
  p = fmaf(p, x, -0.25f);
  p = fmaf(p, x, 1.0f);
  return fmaf(p, x, -0.5772156649f) - logf(x);
}

// x e^x E_1(x) for x >= 1: Hastings' rational approximation as tabulated in
// Abramowitz & Stegun 5.1.56 (absolute error < 2e-8).
__device__ __forceinline__ float xexe1_rational(float x) {
  float num = (((x + 8.5733287401f) * x + 18.0590169730f) * x + 8.6347608925f) * x +
              0.2677737343f;
  float den = (((x + 9.5733223454f) * x + 25.6329561486f) * x + 21.0996530827f) * x +
              3.9584969228f;
  return num / den;
}

__device__ __forceinline__ float e1_dev(float x) {
  return x <= 1.0f ? e1_series(x) : expf(-x) * xexe1_rational(x) / x;
}

// psi(a) = 1 + (a - 1) e^{-a} - a^2 E_1(a)  (Eq. psi).
//  a <= 1: with the series of E_1, psi(a) = Q(a) + a^2 ln a where
//          Q(a) = 1 + (a - 1) e^{-a} + gamma a^2 - a^2 sum_k (-1)^{k+1} a^k/(k k!)
//          is entire; its Taylor coefficients are 2, gamma - 3/2 and
//          (-1)^m 2 / ((m - 2) m!) for m >= 3 (worked out from the two
//          series); eleven terms leave < 4e-10 on [0, 1].
//  1 < a < 15: psi = 1 + e^{-a} [(a - 1) - a (x e^x E_1)(a)] with the
//          rational approximation above (no cancellation).
//  a >= 15: 1 - psi < 2e^{-a}/a < 3e-8, below half an FP32 ulp of 1.
__device__ __forceinline__ float psi_dev(float a) {
  if (a <= 1.0f) {
    if (!(a > 0.0f)) return 0.0f;
    float q = -1.0f / 179625600.0f;
    q = fmaf(q, a, 1.0f / 14515200.0f);
    q = fmaf(q, a, -1.0f / 1270080.0f);
    q = fmaf(q, a, 1.0f / 120960.0f);
    q = fmaf(q, a, -1.0f / 12600.0f);
    q = fmaf(q, a, 1.0f / 1440.0f);
    q = fmaf(q, a, -1.0f / 180.0f);
    q = fmaf(q, a, 1.0f / 24.0f);
    q = fmaf(q, a, -1.0f / 3.0f);
    q = fmaf(q, a, 0.5772156649f - 1.5f);
    q = fmaf(q, a, 2.0f);
    // __logf: absolute error ~2^-21 on ln a near a = 1, i.e. < 2e-7 in a^2 ln a
    return fmaf(a * a, __logf(a), q * a);
  }
  if (a >= 16.0f) return 1.0f;  // 1 - psi(a) < 2 e^{-a}/a < 2^{-25}
  float num = (((a + 8.5733287401f) * a + 18.0590169730f) * a + 8.6347608925f) * a +
              0.2677737343f;
  float den = (((a + 9.5733223454f) * a + 25.6329561486f) * a + 21.0996530827f) * a +
              3.9584969228f;
  return fmaf(__expf(-a), (a - 1.0f) - a * __fdividef(num, den), 1.0f);
}

// psi'(a) = 2 e^{-a} - 2 a E_1(a).
__device__ __forceinline__ float dpsi_dev(float a) {
  if (a <= 1.0f) {
    if (!(a > 0.0f)) return 2.0f;
    return 2.0f * expf(-a) - 2.0f * a * e1_series(a);
  }
  return 2.0f * expf(-a) * (1.0f - xexe1_rational(a));
}

// ------------------------------------------------- packed FP32x2 helpers
// The two species run the same arithmetic on different data; Blackwell's
// packed FP32x2 instructions do both in one issue slot.  Each component is
// rounded exactly as the scalar operation would be.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, f2(-1.0f), a);  // exact: a - b with one rounding
}

// psi at two positive arguments at once.  The lanes of a warp sweep one row
// (the same y) of 32 neighbouring columns, whose mean free paths differ
// little, so with SKIP the two formulas of psi_dev are taken as warp-uniform
// branches: the entire-part series when some lane has an argument <= 1, the
// rational form when some lane has one in (1, 16).  Without SKIP both are
// evaluated and selected (straight-line code that the compiler can
// interleave with the loads of a memory-bound sweep).  At a >= 16,
// 1 - psi(a) < 2 e^{-a}/a < 2^{-25} rounds away and psi = 1.
template <bool SKIP>
__device__ __forceinline__ float2 psi2(float2 a) {
  const bool small = (a.x <= 1.0f) || (a.y <= 1.0f);
  const bool mid = (a.x > 1.0f && a.x < 16.0f) || (a.y > 1.0f && a.y < 16.0f);
  bool do_small = true, do_mid = true;
  if (SKIP) {
    const unsigned lanes = __activemask();
    do_small = __any_sync(lanes, small);
    do_mid = __any_sync(lanes, mid);
  }
  float2 ps = f2(0.0f), pl = f2(1.0f);
  if (do_small) {
    const float2 as = make_float2(fminf(a.x, 1.0f), fminf(a.y, 1.0f));
    float2 q = f2(-1.0f / 179625600.0f);
    q = fma2(q, as, f2(1.0f / 14515200.0f));
    q = fma2(q, as, f2(-1.0f / 1270080.0f));
    q = fma2(q, as, f2(1.0f / 120960.0f));
    q = fma2(q, as, f2(-1.0f / 12600.0f));
    q = fma2(q, as, f2(1.0f / 1440.0f));
    q = fma2(q, as, f2(-1.0f / 180.0f));
    q = fma2(q, as, f2(1.0f / 24.0f));
    q = fma2(q, as, f2(-1.0f / 3.0f));
    q = fma2(q, as, f2(0.5772156649f - 1.5f));
    q = fma2(q, as, f2(2.0f));
    const float2 lg = make_float2(__logf(as.x), __logf(as.y));
    ps = fma2(mul2(as, as), lg, mul2(q, as));
  }
  if (do_mid) {
    // the argument is clamped to [1, 16]: at 16 the formula gives 1 in FP32
    // (1 - psi(16) < 2^-25), and larger arguments cannot overflow it
    const float2 al = make_float2(fminf(fmaxf(a.x, 1.0f), 16.0f), fminf(fmaxf(a.y, 1.0f), 16.0f));
    float2 num = add2(al, f2(8.5733287401f));
    num = fma2(num, al, f2(18.0590169730f));
    num = fma2(num, al, f2(8.6347608925f));
    num = fma2(num, al, f2(0.2677737343f));
    float2 den = add2(al, f2(9.5733223454f));
    den = fma2(den, al, f2(25.6329561486f));
    den = fma2(den, al, f2(21.0996530827f));
    den = fma2(den, al, f2(3.9584969228f));
    const float2 R = make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
    const float2 e = make_float2(__expf(-al.x), __expf(-al.y));
    // 1 + e^{-a} [(a - 1) - a R]
    pl = fma2(e, fma2(make_float2(-al.x, -al.y), R, add2(al, f2(-1.0f))), f2(1.0f));
  }
  // arguments are y / lambda > 0 (y >= 1/2)
  return make_float2(a.x <= 1.0f ? ps.x : pl.x, a.y <= 1.0f ? ps.y : pl.y);
}

// ------------------------------------------------------------- storage
// Populations are stored as deviations d_i = f_i - w_i alpha_si rhobar_s(x)
// from the rest equilibrium (Eq. feq with u = 0) of a fixed per-column
// reference density rhobar_s(x) (the initial profile).  The heavy species'
// rest population carries ~90% of its mass, so storing f_i itself would put
// FP32 rounding of that large number into every moment; the deviations are
// small and keep their full relative precision.  All arithmetic below works
// on deviations relative to the node's own column reference.
template <typename ST>
struct Stor;
// ld/st move one species' value; ld2/st2 move the (a, b) pair of a node's
// population at p (p points at species a, aligned to the pair).
template <>
struct Stor<float> {
  static __device__ __forceinline__ float ld(const float* p) { return __ldg(p); }
  static __device__ __forceinline__ void st(float* p, float v) { *p = v; }
  static __device__ __forceinline__ float2 ld2(const float* p) {
    return __ldg(reinterpret_cast<const float2*>(p));
  }
  static __device__ __forceinline__ void st2(float* p, float2 v) {
    *reinterpret_cast<float2*>(p) = v;
  }
  static __device__ __forceinline__ void st2_sr(float* p, float2 v, unsigned) { st2(p, v); }
};
// Reduced-precision storage of the same deviations: loads widen to FP32, all
// arithmetic is FP32, stores round to nearest.
// Stochastic rounding of an FP32 pair to 16 bits (Blackwell's cvt.rs): each
// value rounds up with probability equal to the fraction of the spacing it
// lies above the lower neighbour, decided by the random bits rbits.  The
// pair is packed with species a (the lower address) in the low half.
__device__ __forceinline__ unsigned cvt_rs_bf16x2(float a, float b, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(b), "f"(a), "r"(rbits));
  return d;
}
__device__ __forceinline__ unsigned cvt_rs_f16x2(float a, float b, unsigned rbits) {
  unsigned d;
  asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(b), "f"(a), "r"(rbits));
  return d;
}

template <>
struct Stor<__nv_bfloat16> {
  static __device__ __forceinline__ float ld(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  static __device__ __forceinline__ void st(__nv_bfloat16* p, float v) {
    *p = __float2bfloat16_rn(v);
  }
  static __device__ __forceinline__ float2 ld2(const __nv_bfloat16* p) {
    return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p)));
  }
  static __device__ __forceinline__ void st2(__nv_bfloat16* p, float2 v) {
    *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v);
  }
  static __device__ __forceinline__ void st2_sr(__nv_bfloat16* p, float2 v, unsigned rbits) {
    *reinterpret_cast<unsigned*>(p) = cvt_rs_bf16x2(v.x, v.y, rbits);
  }
};
template <>
struct Stor<__half> {
  static __device__ __forceinline__ float ld(const __half* p) { return __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(__half* p, float v) { *p = __float2half_rn(v); }
  static __device__ __forceinline__ float2 ld2(const __half* p) {
    return __half22float2(__ldg(reinterpret_cast<const __half2*>(p)));
  }
  static __device__ __forceinline__ void st2(__half* p, float2 v) {
    *reinterpret_cast<__half2*>(p) = __float22half2_rn(v);
  }
  static __device__ __forceinline__ void st2_sr(__half* p, float2 v, unsigned rbits) {
    *reinterpret_cast<unsigned*>(p) = cvt_rs_f16x2(v.x, v.y, rbits);
  }
};

struct Ends {
  float kin[2], kout[2];  // Eq. rho2 density-correction factors
  float gin[2], gout[2];  // ghost reference offsets kappa(2 rb(1) - rb(2)) - rb(0), per species
};

__device__ __forceinline__ unsigned idx(const Lat& L, int sp, int i, int j, int x) {
  return (unsigned)(x >> 5) * L.SS + (unsigned)(j * RS + i * PS + 2 * (x & 31) + sp);
}

// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may start while the kernel before it in the
// stream is still running.  The kernels of the step sequence wait for their
// predecessor's completion and memory (wait) before their first global
// memory access.  The wall kernel lets its successor (the step) launch as
// soon as all of its own CTAs run (launch_dependents); the step kernel does
// so for the instances of a sweep only, and otherwise lets its successor
// launch when it completes.  Launched without the attribute, both
// instructions return at once.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Bulk prefetch of one strip row (all 18 populations of 32 columns, one
// contiguous RS-element run) into L2.  Issued by one lane per warp for the
// row that warp sweeps next, so the DRAM reads of row j + TY are in flight
// while row j is computed, with no registers or shared memory held for them.
template <typename ST>
__device__ __forceinline__ void prefetch_row_l2(const ST* row) {
  static_assert((RS * sizeof(ST)) % 16 == 0, "bulk prefetch size must be a multiple of 16 B");
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(row),
               "r"((int)(RS * sizeof(ST)))
               : "memory");
}

template <typename ST>
__device__ __forceinline__ float ld(const ST* __restrict__ f, const Lat& L, int sp, int i, int j,
                                    int x) {
  return Stor<ST>::ld(f + idx(L, sp, i, j, x));
}

// Deviation (relative to the SOURCE column's reference) that population i
// carries from column xs at row js; the inlet/outlet ghost columns (Eq. rho1,
// all nine populations extrapolated and scaled by Eq. rho2) are virtual.
template <typename ST>
__device__ __forceinline__ float src(const ST* __restrict__ f, const Lat& L, const Ends& E,
                                     float cwi, int sp, int i, int js, int xs) {
  if (!L.x_periodic) {
    if (xs == 0)
      return fmaf(E.kin[sp], 2.0f * ld(f, L, sp, i, js, 1) - ld(f, L, sp, i, js, 2),
                  cwi * E.gin[sp]);
    if (xs == L.Nx - 1)
      return fmaf(E.kout[sp],
                  2.0f * ld(f, L, sp, i, js, L.Nx - 2) - ld(f, L, sp, i, js, L.Nx - 3),
                  cwi * E.gout[sp]);
  }
  return ld(f, L, sp, i, js, xs);
}

// Per-thread column data: own reference density and the reference
// differences to the left and right neighbour columns.
struct ColRef {
  float rb[2], dl[2], dr[2];
};

__device__ __forceinline__ ColRef col_ref(const Lat& L, const float* __restrict__ refrho, int x) {
  ColRef c;
  int xm = x - 1, xp = x + 1;
  if (xm < 0) xm += L.Nx;
  if (xp >= L.Nx) xp -= L.Nx;
  const bool ok = x < L.Nx;
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const float* r = refrho + sp * L.Nx;
    float r0 = ok ? __ldg(r + x) : 0.0f;
    c.rb[sp] = r0;
    c.dl[sp] = ok ? __ldg(r + xm) - r0 : 0.0f;  // exact: adjacent columns differ < 2x
    c.dr[sp] = ok ? __ldg(r + xp) - r0 : 0.0f;
  }
  return c;
}

// Pre-collision deviations of node (x, j): f_i(x) = f'_i(x - c_i) (Eq. MRT)
// re-referenced to column x, with the unknown populations of the wall rows
// from diffuse bounce-back (Eqs. bot, bot2) on the post-collision state of
// the same node.  The wall equilibrium f^eq_i(rho_w, u_w = 0) = w_i s rho_w
// with rho_w from zero normal species flux equals 6 w_i (sum of the outgoing
// f'); its rest part cancels against the reference, leaving
// d_i = (1 - r) d'_opp(i) + r (w_i/(1/6)) sum_outgoing d'.
template <typename ST>
__device__ __forceinline__ void pull_node(const ST* __restrict__ f, const Lat& L, const Ends& E,
                                          const ColRef& C, int x, int j, float2 r_bot2,
                                          float2 r_top2, float fs[2][9]) {
  int xm = x - 1, xp = x + 1;
  if (L.x_periodic) {
    if (xm < 0) xm += L.Nx;
    if (xp >= L.Nx) xp -= L.Nx;
  }
  const bool bot = (j == 0), top = (j == L.N - 1);
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    float* g = fs[sp];
    const float c1 = L.cw1[sp], c5 = L.cw5[sp];
    const float dl = C.dl[sp], dr = C.dr[sp];
    const float r_bot = sp ? r_bot2.y : r_bot2.x, r_top = sp ? r_top2.y : r_top2.x;
    g[0] = ld(f, L, sp, 0, j, x);
    g[1] = fmaf(c1, dl, src(f, L, E, c1, sp, 1, j, xm));
    g[3] = fmaf(c1, dr, src(f, L, E, c1, sp, 3, j, xp));
    if (bot && L.wall_mode == LBM_WALL_BSR) {
      // bounce-back (fraction r) and specular reflection (1 - r): the
      // mirror image of c_5 = (1,1) leaves column x - 1 as c_8, that of c_6
      // leaves column x + 1 as c_7
      const float q = 1.0f - r_bot;
      g[2] = ld(f, L, sp, 4, j, x);
      g[5] = fmaf(r_bot, ld(f, L, sp, 7, j, x), q * fmaf(c5, dl, src(f, L, E, c5, sp, 8, j, xm)));
      g[6] = fmaf(r_bot, ld(f, L, sp, 8, j, x), q * fmaf(c5, dr, src(f, L, E, c5, sp, 7, j, xp)));
    } else if (bot) {
      float o4 = ld(f, L, sp, 4, j, x), o7 = ld(f, L, sp, 7, j, x), o8 = ld(f, L, sp, 8, j, x);
      // the equilibrium parts t/6, t/6 and t - 2 t/6 sum to t exactly up
      // to one rounding, so the wall conserves mass without an FP32 bias
      float t = r_bot * (o4 + o7 + o8), q = 1.0f - r_bot, t6 = t * (1.0f / 6.0f);
      g[2] = fmaf(q, o4, fmaf(-2.0f, t6, t));
      g[5] = fmaf(q, o7, t6);
      g[6] = fmaf(q, o8, t6);
    } else {
      g[2] = ld(f, L, sp, 2, j - 1, x);
      g[5] = fmaf(c5, dl, src(f, L, E, c5, sp, 5, j - 1, xm));
      g[6] = fmaf(c5, dr, src(f, L, E, c5, sp, 6, j - 1, xp));
    }
    if (top && L.wall_mode == LBM_WALL_BSR) {
      // mirror images: c_7 = (-1,-1) of c_6 from column x + 1, c_8 = (1,-1)
      // of c_5 from column x - 1
      const float q = 1.0f - r_top;
      g[4] = ld(f, L, sp, 2, j, x);
      g[7] = fmaf(r_top, ld(f, L, sp, 5, j, x), q * fmaf(c5, dr, src(f, L, E, c5, sp, 6, j, xp)));
      g[8] = fmaf(r_top, ld(f, L, sp, 6, j, x), q * fmaf(c5, dl, src(f, L, E, c5, sp, 5, j, xm)));
    } else if (top) {
      float o2 = ld(f, L, sp, 2, j, x), o5 = ld(f, L, sp, 5, j, x), o6 = ld(f, L, sp, 6, j, x);
      float t = r_top * (o2 + o5 + o6), q = 1.0f - r_top, t6 = t * (1.0f / 6.0f);
      g[4] = fmaf(q, o2, fmaf(-2.0f, t6, t));
      g[7] = fmaf(q, o5, t6);
      g[8] = fmaf(q, o6, t6);
    } else {
      g[4] = ld(f, L, sp, 4, j + 1, x);
      g[7] = fmaf(c5, dr, src(f, L, E, c5, sp, 7, j + 1, xp));
      g[8] = fmaf(c5, dl, src(f, L, E, c5, sp, 8, j + 1, xm));
    }
  }
}

// The same pull for a node whose row is not a wall row and whose strip does
// not contain an end column: nine pair loads (both species) at immediate
// offsets from the row pointers of columns x (p), x - 1 (pl) and x + 1 (pr),
// re-referenced to column x in FP32x2.
template <typename ST>
__device__ __forceinline__ void pull_fast(const ST* __restrict__ p, const ST* __restrict__ pl,
                                          const ST* __restrict__ pr, const Lat& L,
                                          const ColRef& C, float2 g[9]) {
  const float2 dl = make_float2(C.dl[0], C.dl[1]), dr = make_float2(C.dr[0], C.dr[1]);
  g[0] = Stor<ST>::ld2(p);
  g[1] = fma2(L.cw1_2, dl, Stor<ST>::ld2(pl + 1 * PS));
  g[3] = fma2(L.cw1_2, dr, Stor<ST>::ld2(pr + 3 * PS));
  g[2] = Stor<ST>::ld2(p + 2 * PS - RS);
  g[5] = fma2(L.cw5_2, dl, Stor<ST>::ld2(pl + 5 * PS - RS));
  g[6] = fma2(L.cw5_2, dr, Stor<ST>::ld2(pr + 6 * PS - RS));
  g[4] = Stor<ST>::ld2(p + 4 * PS + RS);
  g[7] = fma2(L.cw5_2, dr, Stor<ST>::ld2(pr + 7 * PS + RS));
  g[8] = fma2(L.cw5_2, dl, Stor<ST>::ld2(pl + 8 * PS + RS));
}

// ---------------------------------------------------------------- moments
struct Macro {
  float sd[2];           // sum of deviations: rho_s - rhobar_s
  float rho[2], jx[2], jy[2];
  float ux, uy;
  float n, inv_n, mx;
};

__device__ __forceinline__ void macro(const Lat& L, const ColRef& C, const float fs[2][9],
                                      Macro& m) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const float* g = fs[sp];
    m.sd[sp] = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    m.rho[sp] = C.rb[sp] + m.sd[sp];
    m.jx[sp] = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
    m.jy[sp] = (g[2] - g[4]) + (g[5] - g[7]) + (g[6] - g[8]);
  }
  float rho = m.rho[0] + m.rho[1];
  float inv_rho = __fdividef(1.0f, rho);
  m.ux = (m.jx[0] + m.jx[1]) * inv_rho;
  m.uy = (m.jy[0] + m.jy[1]) * inv_rho;
  m.n = fmaf(m.rho[0], L.s[0], m.rho[1] * L.s[1]);  // number density (Eq. P)
  m.inv_n = __fdividef(1.0f, m.n);
  m.mx = rho * m.inv_n;  // m_x = rho / n
}

// ------------------------------------------- packed per-node arithmetic
// The node update of the step and moments kernels works on g[i] =
// (species a, species b) pairs of the pre-collision deviations.
struct Macro2 {
  float2 sd;   // sum of deviations: rho_s - rhobar_s
  float2 rho;  // species densities
  float2 jx, jy;
  float ux, uy;
  float n, inv_n, mx;
};

__device__ __forceinline__ void macro2(const Lat& L, const ColRef& C, const float2 g[9],
                                       Macro2& m) {
  m.sd = add2(add2(add2(add2(g[0], g[1]), add2(g[2], g[3])), add2(add2(g[4], g[5]), add2(g[6], g[7]))),
              g[8]);
  m.rho = add2(make_float2(C.rb[0], C.rb[1]), m.sd);
  m.jx = add2(add2(sub2(g[1], g[3]), sub2(g[5], g[6])), sub2(g[8], g[7]));
  m.jy = add2(add2(sub2(g[2], g[4]), sub2(g[5], g[7])), sub2(g[6], g[8]));
  const float rho = m.rho.x + m.rho.y;
  const float inv_rho = __fdividef(1.0f, rho);
  m.ux = (m.jx.x + m.jx.y) * inv_rho;
  m.uy = (m.jy.x + m.jy.y) * inv_rho;
  m.n = fmaf(m.rho.x, L.s[0], m.rho.y * L.s[1]);  // number density (Eq. P)
  m.inv_n = __fdividef(1.0f, m.n);
  m.mx = rho * m.inv_n;  // m_x = rho / n
}

// 1/tau_s (Eq. taos) and 1/tau_d (Eq. EQFrsp with lambda_se = lambda_s
// Psi(y; lambda_s), lambda_s = (mu_s/p_s) sqrt(pi k_B T/(2 m_s)), p_s = x_s p),
// with the wall-confinement factor Psi(y) = (psi(y/lambda) + psi((H-y)/lambda))/2
// of the effective mean free path; the six psi values come from three packed
// evaluations.
template <bool SKIP>
__device__ __forceinline__ void rates2(const Lat& L, const Macro2& m, float y, float& om_s,
                                       float& om_d) {
  const float rs_mx = rsqrtf(m.mx);
  const float lam = L.c_lam * m.inv_n * rs_mx;                // mixture mean free path
  const float inv_lam = L.inv_c_lam * m.n * (m.mx * rs_mx);  // 1 / lambda
  const float2 yy = make_float2(y, L.H - y);
  // 1 / lambda_s: n_s / c_xl with the partial pressure, n / c_xl with the
  // mixture pressure
  const float2 ns = mul2(m.rho, L.s2);
  const float2 inv_ls = mul2(L.lam_mix ? f2(m.n) : ns, L.inv_c_xl2);
  const float2 pm = psi2<SKIP>(mul2(yy, f2(inv_lam)));
  const float2 pa = psi2<SKIP>(mul2(yy, f2(inv_ls.x)));
  const float2 pb = psi2<SKIP>(mul2(yy, f2(inv_ls.y)));
  const float ts = lam * (0.5f * (pm.x + pm.y)) * L.c_ts * rs_mx;  // tau_s - 1/2
  om_s = __fdividef(1.0f, 0.5f + ts);
  // x_s lambda_se = c_xl / n * Psi(y; lambda_s) (partial pressure), times
  // x_s = n_s / n with the mixture pressure
  const float2 xs = L.lam_mix ? mul2(ns, f2(m.inv_n)) : f2(1.0f);
  const float2 xle = mul2(mul2(mul2(L.c_xl2, f2(0.5f * m.inv_n)), xs),
                          make_float2(pa.x + pa.y, pb.x + pb.y));
  const float br = rsqrtf(xle.x) + rsqrtf(xle.y);
  // tau_d = 1/2 + c_td / (m_x br^2)  =>  1/tau_d = d / (d/2 + c_td), d = m_x br^2
  const float d = m.mx * br * br;
  om_d = __fdividef(d, fmaf(0.5f, d, L.c_td));
}

// MRT collision of both species at once (Eqs. MR, S, feq) on the deviations g from
// the rest equilibrium of the column reference, in moment space:
// f' = f - M^{-1} S (m - m^eq), M^{-1} = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12,
// 1/6, 1/12, 1/4, 1/4), m^eq = rho_s (1, -4 + 2s + 3u^2, 4 - 3s - 3u^2, u_x,
// -u_x, u_y, -u_y, u_x^2 - u_y^2, u_x u_y).  The reference has m = m^eq(u=0),
// so e - e^eq = sum_i (e_i + 4 - 2s) g_i - 3 rho u^2 and
// eps - eps^eq = sum_i (eps_i - 4 + 3s) g_i + 3 rho u^2 need no large terms
// (ke, kp hold those coefficients for the rest, axis and diagonal classes).
// Returns the x components of the species momenta of Eq. rhou,
// j_x - (j_x - rho_s u_x)/(2 tau_d).
__device__ __forceinline__ float2 collide2(float2 g[9], const Lat& L, float2 rho, float ux,
                                           float uy, float om_e, float om_eps, float om_d,
                                           float om_q, float om_s) {
  const float2 ru2 = mul2(f2(3.0f * (ux * ux + uy * uy)), rho);
  const float2 a14 = add2(add2(g[1], g[2]), add2(g[3], g[4]));
  const float2 a58 = add2(add2(g[5], g[6]), add2(g[7], g[8]));
  const float2 ne =
      fma2(L.ke2[0], g[0], fma2(L.ke2[1], a14, fma2(L.ke2[2], a58, make_float2(-ru2.x, -ru2.y))));
  const float2 neps = fma2(L.kp2[0], g[0], fma2(L.kp2[1], a14, fma2(L.kp2[2], a58, ru2)));
  const float2 d13 = sub2(g[1], g[3]), d24 = sub2(g[2], g[4]);
  const float2 dx56 = add2(sub2(g[5], g[6]), sub2(g[8], g[7]));
  const float2 dy56 = add2(sub2(g[5], g[7]), sub2(g[6], g[8]));
  const float2 jx = add2(d13, dx56);
  const float2 jy = add2(d24, dy56);
  const float2 qx = fma2(f2(-2.0f), d13, dx56);
  const float2 qy = fma2(f2(-2.0f), d24, dy56);
  const float2 pxx = sub2(add2(g[1], g[3]), add2(g[2], g[4]));
  const float2 pxy = sub2(add2(g[5], g[7]), add2(g[6], g[8]));
  const float2 de = mul2(f2(om_e), ne);
  const float2 deps = mul2(f2(om_eps), neps);
  const float2 djx = mul2(f2(om_d), fma2(rho, f2(-ux), jx));
  const float2 djy = mul2(f2(om_d), fma2(rho, f2(-uy), jy));
  const float2 dqx = mul2(f2(om_q), fma2(rho, f2(ux), qx));
  const float2 dqy = mul2(f2(om_q), fma2(rho, f2(uy), qy));
  const float2 dpxx = mul2(f2(om_s), fma2(rho, f2(-(ux * ux - uy * uy)), pxx));
  const float2 dpxy = mul2(f2(om_s), fma2(rho, f2(-(ux * uy)), pxy));
  const float2 c0 = mul2(sub2(de, deps), f2(1.0f / 9.0f));
  const float2 c14 = fma2(de, f2(1.0f / 36.0f), mul2(deps, f2(1.0f / 18.0f)));
  const float2 c58 = fma2(de, f2(-1.0f / 18.0f), mul2(deps, f2(-1.0f / 36.0f)));
  const float2 ax = mul2(sub2(dqx, djx), f2(1.0f / 6.0f));
  const float2 ay = mul2(sub2(dqy, djy), f2(1.0f / 6.0f));
  const float2 bx = fma2(djx, f2(-1.0f / 6.0f), mul2(dqx, f2(-1.0f / 12.0f)));
  const float2 by = fma2(djy, f2(-1.0f / 6.0f), mul2(dqy, f2(-1.0f / 12.0f)));
  const float2 pp = mul2(dpxx, f2(0.25f)), pq = mul2(dpxy, f2(0.25f));
  const float2 u1 = sub2(c14, pp), u2 = add2(c14, pp);  // shared by opposite axis pairs
  const float2 v5 = sub2(c58, pq), v6 = add2(c58, pq);  // and by opposite diagonal pairs
  const float2 w5 = add2(bx, by), w6 = sub2(by, bx);
  g[0] = add2(g[0], c0);
  g[1] = add2(g[1], add2(u1, ax));
  g[3] = add2(g[3], sub2(u1, ax));
  g[2] = add2(g[2], add2(u2, ay));
  g[4] = add2(g[4], sub2(u2, ay));
  g[5] = add2(g[5], add2(v5, w5));
  g[7] = add2(g[7], sub2(v5, w5));
  g[6] = add2(g[6], add2(v6, w6));
  g[8] = add2(g[8], sub2(v6, w6));
  return fma2(f2(-0.5f), djx, jx);
}

// tau_q of Eq. taoq from the wall node's lambda and m_x (tau'_s(0) in its
// last term, dx = 1) and the node's accommodation coefficient (Eq. A12).
__device__ __forceinline__ float tau_q_wall(const Lat& L, const Macro& m, float alpha) {
  const float vs = 0.72360125455f;  // varsigma = sqrt(pi/6)
  float rs_mx = rsqrtf(m.mx);
  float lam = L.c_lam * m.inv_n * rs_mx;
  float g = L.c_ts * rs_mx;  // sqrt(6/(pi m_x))
  float a = L.H / lam;
  float tt = lam * 0.5f * psi_dev(a) * g;
  float dtt = 0.5f * g * (2.0f - dpsi_dev(a));
  float A1 = (2.0f - alpha) / alpha * (1.0f - 0.1817f * alpha);
  float A2 = 1.0f / kPi + 0.5f * A1 * A1;
  return 0.5f + (3.0f + 24.0f * vs * vs * tt * tt * A2) / (16.0f * tt) +
         dtt * (12.0f + 30.0f * tt * vs * A1) / (16.0f * tt * tt);
}

// r of Eq. R, r = 2 - 2/(1 + X), from the mixture molecular mass of the
// reflected post-collision state at the wall node, c_m = c_m0
// (2-alpha)/alpha, for both species: X = c_m sqrt(pi m_x/6) (first printed
// form, the same for both species; masses in units of m_min), c_m sqrt(pi
// m_x/(6 m_s)) (m_min replaced by the species mass) or c_m sqrt(pi m_x^2/(6
// m_s)) (second printed form, m_r = m_s/m_x).  With the BSR wall the
// bounce-back fraction 1/(1 + X) of the same slip factor X.
template <typename ST>
__device__ __forceinline__ float2 dbb_r(const Lat& L, const ColRef& C, const ST* __restrict__ f,
                                        int x, int j, float alpha) {
  float rho[2];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    float acc = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) acc += ld(f, L, sp, i, j, x);
    rho[sp] = C.rb[sp] + acc;
  }
  float mx = (rho[0] + rho[1]) / fmaf(rho[0], L.s[0], rho[1] * L.s[1]);
  float cm = L.c_m0 * (2.0f - alpha) / alpha;
  const float X0 = cm * sqrtf(kPi * mx / 6.0f) * (L.r_form == LBM_R_SECOND ? sqrtf(mx) : 1.0f);
  float r[2];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const float X = L.r_form == LBM_R_FIRST ? X0 : X0 * L.rsqrt_mh[sp];
    r[sp] = L.wall_mode == LBM_WALL_BSR ? 1.0f / (1.0f + X) : 2.0f - 2.0f / (1.0f + X);
  }
  return make_float2(r[0], r[1]);
}

// Density-correction factors of Eq. rho2 for the ghost columns, from the
// column sums of the state being streamed, and the ghost reference offsets;
// only a block whose columns [x0, x0 + width) hold column 1 or column
// N_x - 2 reads them (the others keep kappa = 1, which they never use).
__device__ __forceinline__ Ends load_ends(const Lat& L, const double* __restrict__ cs,
                                          const float* __restrict__ refrho, int x0, int width) {
  Ends E;
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    E.kin[sp] = E.kout[sp] = 1.0f;
    E.gin[sp] = E.gout[sp] = 0.0f;
  }
  if (L.x_periodic) return E;
  const int Nx = L.Nx;
#pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const double* c = cs + (size_t)sp * Nx;
    const float* r = refrho + sp * Nx;
    if (x0 <= 1 && 1 < x0 + width) {
      double k = L.N * L.rho_in[sp] / (2.0 * c[1] - c[2]);
      E.kin[sp] = (float)k;
      E.gin[sp] = (float)(k * (2.0 * (double)r[1] - (double)r[2]) - (double)r[0]);
    }
    if (x0 <= Nx - 2 && Nx - 2 < x0 + width) {
      double k = L.N * L.rho_out[sp] / (2.0 * c[Nx - 2] - c[Nx - 3]);
      E.kout[sp] = (float)k;
      E.gout[sp] = (float)(k * (2.0 * (double)r[Nx - 2] - (double)r[Nx - 3]) - (double)r[Nx - 1]);
    }
  }
  return E;
}

__device__ __forceinline__ bool interior(const Lat& L, int x) {
  return L.x_periodic ? (x < L.Nx) : (x >= 1 && x <= L.Nx - 2);
}

// Per-CTA wall data for the strip: r (both walls), 1/tau_q (both walls).
struct WallSmem {
  float2 r[2][TX];  // (species a, species b) per wall and column
  float om_q[2][TX];
};

// Prologue of the step and moments kernels for the CTA's rows
// [j_begin, j_end): r of a wall is needed only by the CTA that holds that
// wall's row, 1/tau_q of a wall only by CTAs with rows in that wall's half.
// The four tasks run on four warps at once (ty = 0, 1: r of the bottom and
// top wall; ty = 2, 3: their tau_q).  tau_q depends on the wall node's
// pre-collision species densities only (through lambda and m_x), and the
// DBB rule conserves each species' mass at the node whatever r is, so the
// tau_q warps pull the wall node with r = 0 and need not wait for r (the
// BSR rule moves mass between columns: there they evaluate r themselves).
// One wall task of column x: r of wall `wall` (tq false) or 1/tau_q of
// its half (tq true), from the post-collision state fin of the step about
// to run.  Columns outside the interior get r = 1 and 1/tau_q = 1 (unused).
template <typename ST>
__device__ __forceinline__ void wall_task(const Lat& L, const ST* __restrict__ fin,
                                          const float* __restrict__ alpha, const Ends& E,
                                          const ColRef& C, int x, int wall, bool tq, float2& rv,
                                          float& v) {
  v = 1.0f;
  rv = make_float2(1.0f, 1.0f);
  if (!interior(L, x)) return;
  const int jw = wall == 0 ? 0 : L.N - 1;
  const float al = alpha[wall * L.Nx + x];
  if (!tq) {
    rv = dbb_r(L, C, fin, x, jw, al);
  } else {
    float fs[2][9];
    const float2 rr = L.wall_mode == LBM_WALL_BSR ? dbb_r(L, C, fin, x, jw, al)
                                                  : make_float2(0.0f, 0.0f);
    pull_node(fin, L, E, C, x, jw, rr, rr, fs);
    Macro m;
    macro(L, C, fs, m);
    v = 1.0f / tau_q_wall(L, m, al);
  }
}

template <bool WITH_TQ, typename ST>
__device__ __forceinline__ void wall_prologue(const Lat& L, const ST* __restrict__ fin,
                                              const float* __restrict__ alpha, const Ends& E,
                                              const ColRef& C, int x, int j_begin, int j_end,
                                              WallSmem& sm) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  if (ty < (WITH_TQ ? 4 : 2)) {
    const int wall = ty & 1;
    const bool tq = ty >= 2;
    const int half = (L.N + 1) / 2;  // rows j < half use the bottom tau_q
    const bool needed = tq ? (wall == 0 ? j_begin < half : j_end > half)
                           : (wall == 0 ? j_begin == 0 : j_end == L.N);
    float v = 1.0f;
    float2 rv = make_float2(1.0f, 1.0f);
    if (needed) wall_task(L, fin, alpha, E, C, x, wall, tq, rv, v);
    if (tq)
      sm.om_q[wall][tx] = v;
    else
      sm.r[wall][tx] = rv;
  }
  __syncthreads();
}

// The wall tasks of every column as a kernel of their own, ahead of the step
// kernel (16-bit storage, and FP32 grids of several waves): the prologue's
// barrier held the CTA's other warps up while the tau_q warps waited on
// their loads (8 % of the 16-bit step, 4 % of the FP32 step).
// One thread per column and task (blockIdx.y: 0, 1 = r of the bottom, top
// wall; 2, 3 = 1/tau_q of the bottom, top half): r_out [2][Nx] (species
// pair), omq_out [2][Nx].
template <typename ST>
__global__ void __launch_bounds__(128) lbm_walls_kernel(Lat L, const ST* __restrict__ fin,
                                                        const float* __restrict__ refrho,
                                                        const double* __restrict__ cs_in,
                                                        const float* __restrict__ alpha,
                                                        float2* __restrict__ r_out,
                                                        float* __restrict__ omq_out) {
  pdl_launch_dependents();
  pdl_wait();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= L.Nx) return;
  const int wall = blockIdx.y & 1;
  const bool tq = blockIdx.y >= 2;
  const ColRef C = col_ref(L, refrho, x);
  const Ends E = load_ends(L, cs_in, refrho, blockIdx.x * blockDim.x, blockDim.x);
  float2 rv;
  float v;
  wall_task(L, fin, alpha, E, C, x, wall, tq, rv, v);
  if (tq)
    omq_out[wall * L.Nx + x] = v;
  else
    r_out[wall * L.Nx + x] = rv;
}

// Compensated FP32 running sum (Kahan): a thread's partial over its rows of
// one column, accurate to ~1 FP32 ulp of the sum, handed to the FP64 column
// reduction at the end of the sweep (FP64 arithmetic is a slow pipe on this
// part).
struct KahanF {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// ------------------------------------------------------------ step kernel
// Random bits of the stochastic rounding: a 32-bit integer hash (the
// "lowbias32" xorshift-multiply hash of C. Wellons) seeds one linear
// congruential generator per thread and launch (multiplier 1664525 and
// increment 1013904223, the quick generator of Numerical Recipes), whose
// state is folded (high half into the low half) so that both 16-bit halves
// of each word are usable.
__device__ __forceinline__ unsigned hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}
__device__ __forceinline__ unsigned lcg_next(unsigned& s) {
  s = s * 1664525u + 1013904223u;
  return s ^ (s >> 16);
}

template <typename ST>
struct StepArgs {
  const ST* __restrict__ fin;     // post-collision deviations of step t-1
  ST* __restrict__ fout;          // post-collision deviations of step t
  const float* __restrict__ refrho;  // [2][Nx] reference densities
  const double* __restrict__ cs_in;  // [4][Nx] column sums of the state in fin
  double* __restrict__ cs_out;       // [4][Nx] column sums of the state of step t
  const float* __restrict__ alpha;   // [2][Nx]
  double* __restrict__ partials;     // [gridDim.x][NPART]
  unsigned* __restrict__ counter;
  double* __restrict__ diag;         // [DIAG_CAP][NREC]
  unsigned long long* __restrict__ diag_count;
  double* __restrict__ clprof;       // [Nx]
  double* __restrict__ colpart;      // [R][4][Nx] per-row-block column sums (R > 1)
  unsigned* __restrict__ strip_cnt;  // [strips] row blocks finished this step
  int rows_per_block;                // rows of one row block (multiple of TY)
  unsigned seed;                     // 16-bit storage: per-step seed of the
                                     // stochastic rounding; 0 = round to nearest
  // r and 1/tau_q of every column from lbm_walls_kernel ([2][Nx] each,
  // bottom then top), in place of the wall prologue (WK kernels only)
  const float2* __restrict__ wall_r;
  const float* __restrict__ wall_omq;
  // 1: let the next kernel in the stream launch as soon as every CTA of
  // this one runs; 0: when this one completes (see lbm_mix::pdl_early)
  int pdl_early;
};

struct RedSmem {
  double col[4][TY][TX];
  double wsum[TY][6];
  double wmin[TY];
  int wimin[TY];
  int last;
  int last_strip;
};

// Warp-level FP64 sum and (min, argmin) with ties to the smaller column.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ void warp_min(double& v, int& idx) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) {
      v = ov;
      idx = oi;
    }
  }
}

// Column sums -> next step's density correction, C_l(x), per-CTA partials;
// the last CTA to finish reduces the partials in CTA order into one record.
// DIAG = false: only the column sums (the next step's Eq. rho2 input) are
// produced; DIAG = true: also C_l(x), the per-strip partials and the record.
template <bool DIAG, typename ST>
__device__ __forceinline__ void column_epilogue(const Lat& L, const StepArgs<ST>& a, int x,
                                                const double acc[4], RedSmem& rs) {
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * TX + tx;
  const int R = gridDim.y;  // row blocks per strip
#pragma unroll
  for (int k = 0; k < 4; ++k) rs.col[k][ty][tx] = acc[k];
  __syncthreads();
  double c[4];
  if (ty == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double v = 0.0;
      for (int t = 0; t < TY; ++t) v += rs.col[k][t][tx];
      c[k] = v;
    }
  }
  if (R > 1) {
    // Row-block partials of this strip; the last of its R CTAs to finish
    // adds them in row-block order (independent of arrival order).
    if (ty == 0) {
      if (x < L.Nx) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          a.colpart[((size_t)blockIdx.y * 4 + k) * L.Nx + x] = c[k];
      }
      __threadfence();  // the writers publish before the ticket is taken
    }
    __syncthreads();
    if (tid == 0) {
      unsigned ticket = atomicAdd(a.strip_cnt + blockIdx.x, 1u);
      rs.last_strip = (ticket == (unsigned)R - 1u);
    }
    __syncthreads();
    if (!rs.last_strip) return;
    if (ty == 0) {
      __threadfence();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        double v = 0.0;
        if (x < L.Nx)
          for (int r = 0; r < R; ++r) v += __ldcg(a.colpart + ((size_t)r * 4 + k) * L.Nx + x);
        c[k] = v;
      }
      if (tx == 0) a.strip_cnt[blockIdx.x] = 0u;
    }
  }
  if (!DIAG) {
    if (ty == 0 && x < L.Nx) {
#pragma unroll
      for (int k = 0; k < 4; ++k) a.cs_out[(size_t)k * L.Nx + x] = c[k];
    }
    return;
  }
  if (ty == 0) {
    const bool in = interior(L, x);
    if (x < L.Nx) {
#pragma unroll
      for (int k = 0; k < 4; ++k) a.cs_out[(size_t)k * L.Nx + x] = c[k];
    }
    double Cl = 0.0;
    if (in) {
      double na = c[0] * L.s[0], nb = c[1] * L.s[1];
      Cl = (L.light == 0 ? na : nb) / (na + nb);
      a.clprof[x] = Cl;
    } else if (x < L.Nx) {
      a.clprof[x] = (x == 0) ? L.C_in : L.C_out;
    }
    double vmin = in ? Cl : INFINITY;
    int imin = in ? x : 0x7fffffff;
    warp_min(vmin, imin);
    double p_dev = warp_sum(in ? Cl - L.C_in : 0.0);
    double p_ma = warp_sum(in ? c[2] : 0.0);
    double p_mb = warp_sum(in ? c[3] : 0.0);
    double p_ra = warp_sum(in ? c[0] : 0.0);
    double p_rb = warp_sum(in ? c[1] : 0.0);
    double p_n = warp_sum(in ? 1.0 : 0.0);
    if (tx == 0) {
      double* p = a.partials + (size_t)blockIdx.x * NPART;
      p[0] = vmin;
      p[1] = (double)imin;
      p[2] = p_dev;
      p[3] = p_ma;
      p[4] = p_mb;
      p[5] = p_ra;
      p[6] = p_rb;
      p[7] = p_n;
      __threadfence();
    }
  }
  __syncthreads();
  if (tid == 0) {
    unsigned ticket = atomicAdd(a.counter, 1u);
    rs.last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!rs.last) return;
  __threadfence();
  // Last CTA: every thread folds a fixed subset of the partials in CTA order,
  // then a fixed shuffle tree per warp and warp order in thread 0, so the
  // result does not depend on which CTA finished last.
  const int nt = TX * TY;
  double vmin = INFINITY, sm[6] = {0, 0, 0, 0, 0, 0};
  int imin = 0x7fffffff;
  for (int b = tid; b < (int)gridDim.x; b += nt) {
    const double* p = a.partials + (size_t)b * NPART;
    double v = __ldcg(p + 0);
    int i = (int)__ldcg(p + 1);
    if (v < vmin || (v == vmin && i < imin)) {
      vmin = v;
      imin = i;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) sm[k] += __ldcg(p + 2 + k);
  }
  warp_min(vmin, imin);
#pragma unroll
  for (int k = 0; k < 6; ++k) sm[k] = warp_sum(sm[k]);
  const int lane = tid & 31, wid = tid >> 5;
  if (lane == 0) {
    rs.wmin[wid] = vmin;
    rs.wimin[wid] = imin;
#pragma unroll
    for (int k = 0; k < 6; ++k) rs.wsum[wid][k] = sm[k];
  }
  __syncthreads();
  if (tid == 0) {
    double tot[6] = {0, 0, 0, 0, 0, 0};
    double mn = INFINITY;
    int im = 0x7fffffff;
    for (int w = 0; w < nt / 32; ++w) {
      for (int k = 0; k < 6; ++k) tot[k] += rs.wsum[w][k];
      if (rs.wmin[w] < mn || (rs.wmin[w] == mn && rs.wimin[w] < im)) {
        mn = rs.wmin[w];
        im = rs.wimin[w];
      }
    }
    double dev = tot[0];
    if (!L.x_periodic) dev += (L.C_out - L.C_in);  // the outlet boundary column
    const double ncol = tot[5];
    unsigned long long cnt = *a.diag_count + 1ull;
    double* rec = a.diag + (size_t)((cnt - 1ull) % DIAG_CAP) * NREC;
    rec[0] = (double)cnt;
    rec[1] = (L.C_in - mn) / L.C_in;
    rec[2] = dev / ((double)L.Nx * L.C_in);
    rec[3] = tot[1] / ncol;
    rec[4] = tot[2] / ncol;
    rec[5] = (double)im;
    rec[6] = tot[3];
    rec[7] = tot[4];
    *a.diag_count = cnt;
    *a.counter = 0u;
    __threadfence();
  }
}

// DIAG: reduce the separation diagnostics of the new state (every
// diag_every-th step); otherwise only the strips holding the end columns
// reduce the column sums the next step's density correction needs.
// WK: r and 1/tau_q of the columns come from lbm_walls_kernel, launched
// ahead of the step (always with 16-bit storage), instead of the CTA's wall
// prologue.
template <typename ST, bool DIAG, bool WK = (sizeof(ST) < 4)>
__global__ void __launch_bounds__(TX* TY, 3) lbm_step_kernel(Lat L, StepArgs<ST> a) {
  __shared__ WallSmem wsm;
  __shared__ RedSmem rsm;
  if (a.pdl_early) pdl_launch_dependents();
  pdl_wait();
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x0 = blockIdx.x * TX, x = x0 + tx;
  const ColRef C = col_ref(L, a.refrho, x);
  const Ends E = load_ends(L, a.cs_in, a.refrho, blockIdx.x * TX, TX);
  const int j_begin = blockIdx.y * a.rows_per_block;
  const int j_end = min(L.N, j_begin + a.rows_per_block);
  // the first row of each warp is on its way into L2 while the wall prologue
  // (if any) runs
  if (tx == 0 && j_begin + ty < j_end)
    prefetch_row_l2(a.fin + (size_t)blockIdx.x * L.SS + (size_t)(j_begin + ty) * RS);
  // r and 1/tau_q of this column: from lbm_walls_kernel (WK, read where they
  // are used) or from the CTA's wall prologue
  const int xc = x < L.Nx ? x : L.Nx - 1;
  if constexpr (!WK) wall_prologue<true>(L, a.fin, a.alpha, E, C, x, j_begin, j_end, wsm);
  auto wall_r = [&](int w) -> float2 {
    if constexpr (WK) return a.wall_r[w * L.Nx + xc];
    else return wsm.r[w][tx];
  };
  auto wall_omq = [&](int h) -> float {
    if constexpr (WK) return a.wall_omq[h * L.Nx + xc];
    else return wsm.om_q[h][tx];
  };
  const bool in = interior(L, x);
  // strips holding column 1 or N_x - 2 take the general pull (ghost columns)
  const bool edge_strip = !L.x_periodic && (x0 <= 1 || x0 + TX > L.Nx - 2);
  int xm = x - 1, xp = x + 1;
  if (xm < 0) xm += L.Nx;
  if (xp >= L.Nx) xp -= L.Nx;
  const unsigned base = blockIdx.x * L.SS + 2 * tx;  // row 0, i = 0, species a of column x
  const int offl = (int)(idx(L, 0, 0, 0, xm) - base), offr = (int)(idx(L, 0, 0, 0, xp) - base);
  const int half = (L.N + 1) / 2;  // rows j < half (1-based 2J <= N+1) use the bottom tau_q
  KahanF acc[4];
  const bool reduce = DIAG || edge_strip;
  // per-thread generator of the stochastic rounding (16-bit storage only)
  unsigned rng = sizeof(ST) < 4
                     ? hash32(a.seed ^ hash32((blockIdx.y * gridDim.x + blockIdx.x) * (TX * TY) +
                                             ty * TX + tx))
                     : 0u;
  if (in) {
    for (int j = j_begin + ty; j < j_end; j += TY) {
      float2 g[9];
      const ST* p = a.fin + base + j * RS;
      // row start is 16-byte aligned (RS * sizeof(ST) is a multiple of 16);
      // the prefetched row lies inside this strip (j + TY < j_end <= N)
      if (tx == 0 && j + TY < j_end) prefetch_row_l2(p + TY * RS);
      if (!edge_strip && j != 0 && j != L.N - 1) {
        pull_fast(p, p + offl, p + offr, L, C, g);
      } else {
        float fs[2][9];
        pull_node(a.fin, L, E, C, x, j, wall_r(0), wall_r(1), fs);
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = make_float2(fs[0][i], fs[1][i]);
      }
      Macro2 m;
      macro2(L, C, g, m);
      float om_s, om_d;
      // 16-bit storage halves the bytes and leaves the sweep bound by
      // instruction issue: there skipping psi work pays, for FP32 it does not
      rates2<(sizeof(ST) < 4)>(L, m, (float)j + 0.5f, om_s, om_d);
      const float om_q = wall_omq(j < half ? 0 : 1);
      const float2 mxs =
          collide2(g, L, m.rho, m.ux, m.uy, L.om_e, L.om_eps, om_d, om_q, om_s);
      if (reduce) {
        acc[0].add(m.sd.x);
        acc[1].add(m.sd.y);
        acc[2].add(mxs.x);
        acc[3].add(mxs.y);
      }
      ST* o = a.fout + base + j * RS;
      if (sizeof(ST) < 4 && a.seed != 0u) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Stor<ST>::st2_sr(o + i * PS, g[i], lcg_next(rng));
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) Stor<ST>::st2(o + i * PS, g[i]);
      }
    }
  }
  if (!reduce) return;  // CTA-uniform
  // column sum of rho_s = N rhobar_s + sum of deviations; the reference part
  // is added once per column (by the ty = 0 thread of the first row block)
  const bool adds_ref = in && ty == 0 && blockIdx.y == 0;
  double accd[4];
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
    accd[sp] = (adds_ref ? (double)L.N * (double)C.rb[sp] : 0.0) + acc[sp].value();
  accd[2] = acc[2].value();
  accd[3] = acc[3].value();
  column_epilogue<DIAG>(L, a, x, accd, rsm);
}

// ---------------------------------------------------------- moments kernel
// Fields of the state obtained by streaming fin (direct = 0), or of fin
// itself (direct = 1), FP64 [6][N][Nx]: rho_a, rho_b, u_a (x, y), u_b (x, y)
// with the species momentum of Eq. rhou.
template <typename ST>
__global__ void __launch_bounds__(TX* TY)
    lbm_moments_kernel(Lat L, const ST* __restrict__ fin, const float* __restrict__ refrho,
                       const double* __restrict__ cs_in, const float* __restrict__ alpha,
                       int direct, double* __restrict__ out) {
  __shared__ WallSmem wsm;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * TX + tx;
  const ColRef C = col_ref(L, refrho, x);
  const Ends E = load_ends(L, cs_in, refrho, blockIdx.x * TX, TX);
  if (!direct) wall_prologue<false>(L, fin, alpha, E, C, x, 0, L.N, wsm);
  if (!interior(L, x)) return;
  const size_t plane = (size_t)L.N * L.Nx;
  for (int j = ty; j < L.N; j += TY) {
    float fs[2][9];
    if (direct) {
#pragma unroll
      for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int i = 0; i < 9; ++i) fs[sp][i] = ld(fin, L, sp, i, j, x);
    } else {
      pull_node(fin, L, E, C, x, j, wsm.r[0][tx], wsm.r[1][tx], fs);
    }
    float2 g[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = make_float2(fs[0][i], fs[1][i]);
    Macro2 m;
    macro2(L, C, g, m);
    float om_s, om_d;
    rates2<false>(L, m, (float)j + 0.5f, om_s, om_d);
    // Eq. rhou: (2 tau_d - 1)/(2 tau_d) = 1 - om_d/2, 1/(2 tau_d) = om_d/2
    const float w1 = 1.0f - 0.5f * om_d, w2 = 0.5f * om_d;
    const size_t o = (size_t)j * L.Nx + x;
    const float rho_s[2] = {m.rho.x, m.rho.y}, sd[2] = {m.sd.x, m.sd.y};
    const float jxs[2] = {m.jx.x, m.jx.y}, jys[2] = {m.jy.x, m.jy.y};
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      float mx = fmaf(w1, jxs[sp], w2 * rho_s[sp] * m.ux);
      float my = fmaf(w1, jys[sp], w2 * rho_s[sp] * m.uy);
      out[sp * plane + o] = (double)C.rb[sp] + (double)sd[sp];
      out[(2 + 2 * sp) * plane + o] = (double)(mx / rho_s[sp]);
      out[(3 + 2 * sp) * plane + o] = (double)(my / rho_s[sp]);
    }
  }
}

// Boundary columns of the moment fields (pressure ends): rho_s =
// kappa_s (2 rho_s(1) - rho_s(2)) with kappa_s of Eq. rho2, u_s linearly
// extrapolated.  Block 0: inlet, block 1: outlet.
__global__ void lbm_moments_ends_kernel(Lat L, double* __restrict__ out) {
  __shared__ double red[2][256];
  const int end = blockIdx.x, tid = threadIdx.x;
  const int xb = end == 0 ? 0 : L.Nx - 1, x1 = end == 0 ? 1 : L.Nx - 2,
            x2 = end == 0 ? 2 : L.Nx - 3;
  const size_t plane = (size_t)L.N * L.Nx;
  double sa = 0.0, sb = 0.0;
  for (int j = tid; j < L.N; j += blockDim.x) {
    size_t o = (size_t)j * L.Nx;
    sa += 2.0 * out[o + x1] - out[o + x2];
    sb += 2.0 * out[plane + o + x1] - out[plane + o + x2];
  }
  red[0][tid] = sa;
  red[1][tid] = sb;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) {
      red[0][tid] += red[0][tid + w];
      red[1][tid] += red[1][tid + w];
    }
    __syncthreads();
  }
  const double* tgt = end == 0 ? L.rho_in : L.rho_out;
  const double ka = L.N * tgt[0] / red[0][0], kb = L.N * tgt[1] / red[1][0];
  for (int j = tid; j < L.N; j += blockDim.x) {
    size_t o = (size_t)j * L.Nx;
    out[o + xb] = ka * (2.0 * out[o + x1] - out[o + x2]);
    out[plane + o + xb] = kb * (2.0 * out[plane + o + x1] - out[plane + o + x2]);
    for (int k = 2; k < 6; ++k)
      out[k * plane + o + xb] = 2.0 * out[k * plane + o + x1] - out[k * plane + o + x2];
  }
}

// ------------------------------------------------------------ init kernels
// Column sums of a state: sum_j rho_s = N rhobar_s + sum_j sum_i d_i and the
// raw x momenta, used as the density-correction input of the first step
// after init or a state upload.
template <typename ST>
__global__ void lbm_colsum_kernel(Lat L, const ST* __restrict__ f,
                                  const float* __restrict__ refrho, double* __restrict__ cs) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= L.Nx) return;
  for (int sp = 0; sp < 2; ++sp) {
    double r = 0.0, m = 0.0;
    for (int j = 0; j < L.N; ++j) {
      float v[9];
      for (int i = 0; i < 9; ++i) v[i] = ld(f, L, sp, i, j, x);
      r += (double)(((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8]);
      m += (double)((v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]));
    }
    cs[(size_t)sp * L.Nx + x] = (double)L.N * (double)refrho[sp * L.Nx + x] + r;
    cs[(size_t)(2 + sp) * L.Nx + x] = m;
  }
}

// Re-referencing: new reference rhobar'_s(x) = cs[s][x] / N (the column
// mean of the current state) for the updated columns, unchanged elsewhere;
// d_i <- d_i + w_i alpha_si (rhobar_s - rhobar'_s) in place, in both
// buffers (the moments of the current step are formed by streaming the
// previous one).  One thread per (x, j), both species of a population as
// one pair.
template <typename ST>
__global__ void lbm_reref_kernel(Lat L, ST* __restrict__ f, ST* __restrict__ f_prev,
                                 const float* __restrict__ ref_old,
                                 const double* __restrict__ cs, float* __restrict__ ref_new) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (x >= L.Nx) return;
  float2 ro = make_float2(ref_old[x], ref_old[L.Nx + x]), rn = ro;
  if (interior(L, x))
    rn = make_float2((float)(cs[x] / L.N), (float)(cs[L.Nx + x] / L.N));
  if (j == 0) {
    ref_new[x] = rn.x;
    ref_new[L.Nx + x] = rn.y;
  }
  const float2 dr = sub2(ro, rn);
  ST* p = f + idx(L, 0, 0, j, x);
  ST* q = f_prev + idx(L, 0, 0, j, x);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float2 cw = i == 0 ? make_float2(L.cw0[0], L.cw0[1])
                             : (i < 5 ? L.cw1_2 : L.cw5_2);
    Stor<ST>::st2(p + i * PS, fma2(cw, dr, Stor<ST>::ld2(p + i * PS)));
    Stor<ST>::st2(q + i * PS, fma2(cw, dr, Stor<ST>::ld2(q + i * PS)));
  }
}

// Full populations <-> stored deviations.  to_dev = 1: reads f from `in`
// (FP32, unpadded [2][9][N][Nx]) and stores d = f - ref in the strip layout;
// to_dev = 0: writes f = d + ref to `out` (T = float or double, unpadded).
template <typename ST, typename T>
__global__ void lbm_convert_kernel(Lat L, ST* __restrict__ f, const float* __restrict__ refrho,
                                   int to_dev, const float* __restrict__ in, T* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y, sp = blockIdx.z;
  if (x >= L.Nx) return;
  const float rb = refrho[sp * L.Nx + x];
  for (int i = 0; i < 9; ++i) {
    const float cw = i == 0 ? L.cw0[sp] : (i < 5 ? L.cw1[sp] : L.cw5[sp]);
    const float ref = cw * rb;
    ST* p = f + idx(L, sp, i, j, x);
    const size_t h = (((size_t)sp * 9 + i) * L.N + j) * L.Nx + x;
    if (to_dev)
      Stor<ST>::st(p, in[h] - ref);
    else
      out[h] = (T)Stor<ST>::ld(p) + (T)ref;
  }
}

// Volume flow through column x: sum over the rows of the mixture velocity
// u_x = (rho_a u_a,x + rho_b u_b,x) / (rho_a + rho_b) of a moments array
// [6][N][Nx] (rho_a, rho_b, u_a (x, y), u_b (x, y)); one block, fixed order.
__global__ void lbm_volume_flow_kernel(const double* __restrict__ mom, int N, int Nx, int x,
                                       double* __restrict__ out) {
  __shared__ double red[256];
  const size_t plane = (size_t)N * Nx;
  double v = 0.0;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const size_t o = (size_t)j * Nx + x;
    const double ra = mom[o], rb = mom[plane + o];
    v += (ra * mom[2 * plane + o] + rb * mom[4 * plane + o]) / (ra + rb);
  }
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) s += red[k];
    *out = s;
  }
}

// Steady-state residual over the column sums: R = |c - c_old| / (K |c|),
// then c_old = c.  One CTA.
__global__ void lbm_residual_kernel(const double* __restrict__ c, double* __restrict__ c_old,
                                    long n, double K, int have_old, double* __restrict__ R) {
  __shared__ double s1[32], s2[32];
  double d2 = 0.0, c2 = 0.0;
  for (long k = threadIdx.x; k < n; k += blockDim.x) {
    double v = c[k];
    double d = v - c_old[k];
    d2 += d * d;
    c2 += v * v;
    c_old[k] = v;
  }
  d2 = warp_sum(d2);
  c2 = warp_sum(c2);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s1[wid] = d2;
    s2[wid] = c2;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    d2 = lane < nw ? s1[lane] : 0.0;
    c2 = lane < nw ? s2[lane] : 0.0;
    d2 = warp_sum(d2);
    c2 = warp_sum(c2);
    if (lane == 0) *R = have_old ? sqrt(d2) / (K * sqrt(c2)) : INFINITY;
  }
}

__global__ void lbm_special_kernel(const double* __restrict__ x, double* __restrict__ e1,
                                   double* __restrict__ ps, long n) {
  long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  float v = (float)x[k];
  e1[k] = (double)e1_dev(v);
  ps[k] = (double)psi_dev(v);
}

}  // namespace

// ================================================================ host API
struct lbm_mix {
  lbm_mix_params p;
  Lat L;
  int device;
  int nsm;            // streaming multiprocessors of the device
  cudaStream_t stream;
  bool own_stream;
  int nblocks;
  void* buf[2];       // post-collision deviations, A/B (element type per storage)
  size_t elem;        // bytes per stored population
  float* refrho;      // [2][Nx] reference densities rhobar_s(x)
  float* refrho_alt;  // the next reference table of lbm_mix_rereference
  double* cs_tmp;     // [4][Nx] column sums of lbm_mix_rereference
  float* scratch;     // full-population staging for get_post_state (lazy)
  double* cs[2];
  double* cs_snap;
  float* alpha;
  double* partials;
  unsigned* counter;
  double* diag;
  unsigned long long* diag_count;
  double* clprof;
  float2* wall_r;      // [2][Nx] r per wall and column (lbm_walls_kernel)
  float* wall_omq;     // [2][Nx] 1/tau_q per half and column (lbm_walls_kernel)
  double* colpart;     // [R][4][Nx]
  unsigned* strip_cnt; // [nblocks]
  int R, rows_per_block;
  int R_alloc;        // row blocks colpart has room for
  double* resid;
  double* mom;
  double* h_pinned;  // small pinned staging area
  // The step kernel lets the next kernel launch as soon as all of its CTAs
  // run (instances of a sweep, whose streams compete for the SMs: the sweep
  // took 57.9 instead of 60.1 s), or only when it completes (lone handles:
  // the next kernel's CTAs are then spread over the SMs the step frees;
  // 0.2197 instead of 0.2235 s for 5000 steps of a 1280 x 64 channel).
  bool pdl_early;
  int cur;           // buffer holding the latest post-collision state
  long steps;
  bool have_snap;
};

namespace {

int validate(const lbm_mix_params* p, int* Nx_out) {
  if (!p) return set_err(LBM_EINVAL, "params is NULL");
  if (!(p->m_a > 0 && p->m_b > 0 && isfinite(p->m_a) && isfinite(p->m_b)))
    return set_err(LBM_EINVAL, "masses must be positive and finite");
  if (!(p->C_l > 0 && p->C_l < 1)) return set_err(LBM_EINVAL, "C_l must be in (0,1)");
  if (p->C_l_out >= 0 && !(p->C_l_out > 0 && p->C_l_out < 1))
    return set_err(LBM_EINVAL, "C_l_out must be in (0,1) or negative");
  if (!(p->theta >= 1.0 && isfinite(p->theta))) return set_err(LBM_EINVAL, "theta must be >= 1");
  if (!(p->Kn_out > 0 && isfinite(p->Kn_out))) return set_err(LBM_EINVAL, "Kn_out must be > 0");
  if (p->N < 2) return set_err(LBM_EINVAL, "N must be >= 2");
  long Nx = p->N_x;
  if (Nx <= 0) {
    if (!(p->L_over_H > 0 && isfinite(p->L_over_H)))
      return set_err(LBM_EINVAL, "L_over_H must be > 0 when N_x <= 0");
    Nx = lround(p->N * p->L_over_H);
  }
  if (Nx < 4) return set_err(LBM_EINVAL, "need N_x >= 4 columns (got %ld)", Nx);
  if (!(p->accommodation > 0 && p->accommodation <= 1))
    return set_err(LBM_EINVAL, "accommodation must be in (0,1]");
  if (!(p->c_m0 >= 0 && isfinite(p->c_m0))) return set_err(LBM_EINVAL, "c_m0 must be >= 0");
  if (!(p->tau_rho > 0.5 && p->tau_e > 0.5 && p->tau_eps > 0.5))
    return set_err(LBM_EINVAL, "tau_rho, tau_e, tau_eps must exceed 1/2");
  if (!(p->mu_ratio_a > 0 && p->mu_ratio_b > 0))
    return set_err(LBM_EINVAL, "viscosity ratios must be > 0");
  if (p->storage != LBM_FP32 && p->storage != LBM_BF16 && p->storage != LBM_FP16)
    return set_err(LBM_EINVAL, "storage must be LBM_FP32, LBM_BF16 or LBM_FP16");
  if (p->x_periodic != 0 && p->x_periodic != 1) return set_err(LBM_EINVAL, "x_periodic is 0 or 1");
  if (p->diag_every < 1) return set_err(LBM_EINVAL, "diag_every must be >= 1");
  if (p->reref_every < -1) return set_err(LBM_EINVAL, "reref_every must be >= -1");
  if (p->r_form != LBM_R_FIRST && p->r_form != LBM_R_SPECIES && p->r_form != LBM_R_SECOND)
    return set_err(LBM_EINVAL, "r_form must be LBM_R_FIRST, LBM_R_SPECIES or LBM_R_SECOND");
  if (p->lambda_pressure != 0 && p->lambda_pressure != 1)
    return set_err(LBM_EINVAL, "lambda_pressure must be 0 (partial) or 1 (mixture)");
  if (p->wall != LBM_WALL_DBB && p->wall != LBM_WALL_BSR)
    return set_err(LBM_EINVAL, "wall must be LBM_WALL_DBB or LBM_WALL_BSR");
  if (p->rounding != LBM_ROUND_STOCHASTIC && p->rounding != LBM_ROUND_NEAREST)
    return set_err(LBM_EINVAL, "rounding must be LBM_ROUND_STOCHASTIC or LBM_ROUND_NEAREST");
  long pitch = (Nx + 31) / 32 * 32;
  double elems = 18.0 * (double)p->N * (double)pitch;
  if (elems >= 2147483648.0)
    return set_err(LBM_EINVAL, "lattice too large: 18*N*pitch must stay below 2^31");
  *Nx_out = (int)Nx;
  return LBM_OK;
}

// Lattice constants in the units of the header (k_B T = 1/3, m_min = 1,
// outlet number density 1), derived in FP64.
Lat derive(const lbm_mix_params* p, int Nx) {
  Lat L;
  memset(&L, 0, sizeof L);
  const double PI = 3.14159265358979323846;
  L.N = p->N;
  L.Nx = Nx;
  L.pitch = (Nx + 31) / 32 * 32;
  L.SS = (unsigned)((long)L.N * RS);
  L.x_periodic = p->x_periodic;
  L.wall_mode = p->wall;
  L.r_form = p->r_form;
  L.lam_mix = p->lambda_pressure;
  double m_min = fmin(p->m_a, p->m_b);
  double mh[2] = {p->m_a / m_min, p->m_b / m_min};
  L.light = (p->m_a <= p->m_b) ? 0 : 1;
  double Cin = p->C_l, Cout = p->C_l_out < 0 ? p->C_l : p->C_l_out;
  double Ci[2], Co[2];
  Ci[L.light] = Cin;
  Ci[1 - L.light] = 1.0 - Cin;
  Co[L.light] = Cout;
  Co[1 - L.light] = 1.0 - Cout;
  L.C_in = Cin;
  L.C_out = Cout;
  double mx_out = Co[0] * mh[0] + Co[1] * mh[1];
  double lam_out = p->Kn_out * p->N;
  // lambda = (mu / p) sqrt(pi k_B T / (2 m_x)) with p_out = 1/3 at the outlet
  double mu = lam_out * (1.0 / 3.0) / sqrt(PI / (6.0 * mx_out));
  double mu_s[2] = {p->mu_ratio_a * mu, p->mu_ratio_b * mu};
  for (int sp = 0; sp < 2; ++sp) {
    L.s[sp] = (float)(1.0 / mh[sp]);
    L.cw0[sp] = (float)((9.0 - 5.0 * (double)L.s[sp]) / 9.0);
    L.cw1[sp] = (float)((double)L.s[sp] / 9.0);
    L.cw5[sp] = (float)((double)L.s[sp] / 36.0);
    const float sf = L.s[sp];
    L.ke[sp][0] = -2.0f * sf;
    L.ke[sp][1] = 3.0f - 2.0f * sf;
    L.ke[sp][2] = 6.0f - 2.0f * sf;
    L.kp[sp][0] = 3.0f * sf;
    L.kp[sp][1] = 3.0f * sf - 6.0f;
    L.kp[sp][2] = 3.0f * sf - 3.0f;
  }
  for (int sp = 0; sp < 2; ++sp) {
    float* s2 = &L.s2.x;
    s2[sp] = L.s[sp];
    (&L.cw1_2.x)[sp] = L.cw1[sp];
    (&L.cw5_2.x)[sp] = L.cw5[sp];
    for (int k = 0; k < 3; ++k) {
      (&L.ke2[k].x)[sp] = L.ke[sp][k];
      (&L.kp2[k].x)[sp] = L.kp[sp][k];
    }
    L.mh[sp] = mh[sp];
    L.rsqrt_mh[sp] = (float)(1.0 / sqrt(mh[sp]));
    double cxl = 3.0 * mu_s[sp] * sqrt(PI / (6.0 * mh[sp]));
    L.c_xl[sp] = (float)cxl;
    L.inv_c_xl[sp] = (float)(1.0 / cxl);
    (&L.c_xl2.x)[sp] = L.c_xl[sp];
    (&L.inv_c_xl2.x)[sp] = L.inv_c_xl[sp];
    L.rho_in[sp] = p->theta * Ci[sp] * mh[sp];
    L.rho_out[sp] = Co[sp] * mh[sp];
  }
  double clam = 3.0 * mu * sqrt(PI / 6.0);
  L.c_lam = (float)clam;
  L.inv_c_lam = (float)(1.0 / clam);
  L.c_ts = (float)sqrt(6.0 / PI);
  L.c_td = (float)(1.5 * sqrt(3.0 * (mh[0] + mh[1]) * mh[0] * mh[1] / 1.0));
  L.om_e = (float)(1.0 / p->tau_e);
  L.om_eps = (float)(1.0 / p->tau_eps);
  L.c_m0 = (float)p->c_m0;
  L.H = (float)p->N;
  return L;
}

// Host copy of the step kernel's seed hash (lowbias32).
unsigned host_hash32(unsigned x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// Rows of one strip per CTA of the step kernel unless the caller sets a
// schedule: measured on GB300 against 64 ... 512 rows, 96 is within 1 % of
// the best on the 32768 x 512 and 16384 x 256 channels (128 rows: 2 % and
// 11 % slower; 512: 30 % slower).
constexpr int DEFAULT_ROWS = 96;
int default_rows(int N) {
  const int n8 = (N + TY - 1) / TY * TY;
  return n8 < DEFAULT_ROWS ? n8 : DEFAULT_ROWS;
}

// Calls f(type tag) with the storage element type of the handle.
template <typename F>
int with_storage(const lbm_mix* h, F&& f) {
  switch (h->p.storage) {
    case LBM_FP32: return f(float());
    case LBM_BF16: return f(__nv_bfloat16());
    case LBM_FP16: return f(__half());
    default: return set_err(LBM_EINVAL, "unknown storage %d", h->p.storage);
  }
}

int launch_colsum(lbm_mix* h, int b) {
  return with_storage(h, [&](auto tag) -> int {
    using ST = decltype(tag);
    dim3 blk(128), grd((h->L.Nx + 127) / 128);
    lbm_colsum_kernel<ST><<<grd, blk, 0, h->stream>>>(h->L, (const ST*)h->buf[b], h->refrho,
                                                      h->cs[b]);
    CK(cudaGetLastError());
    return LBM_OK;
  });
}

// Column sums of the current state into cs_tmp, then the in-place rewrite
// of the deviations against the new column means; the reference tables swap.
int rereference(lbm_mix* h) {
  const int b = h->cur;
  int st = with_storage(h, [&](auto tag) -> int {
    using ST = decltype(tag);
    dim3 blk(128), grd((h->L.Nx + 127) / 128);
    lbm_colsum_kernel<ST><<<grd, blk, 0, h->stream>>>(h->L, (const ST*)h->buf[b], h->refrho,
                                                      h->cs_tmp);
    CK(cudaGetLastError());
    dim3 grd2((h->L.Nx + 127) / 128, h->L.N);
    lbm_reref_kernel<ST><<<grd2, blk, 0, h->stream>>>(h->L, (ST*)h->buf[b], (ST*)h->buf[1 - b],
                                                      h->refrho, h->cs_tmp, h->refrho_alt);
    CK(cudaGetLastError());
    return LBM_OK;
  });
  if (st) return st;
  float* t = h->refrho;
  h->refrho = h->refrho_alt;
  h->refrho_alt = t;
  return LBM_OK;
}

// Steady-state residual of the last k steps (Sec. 4 convergence check, over
// the column sums of the latest DIAG step) into h->h_pinned[0], async.
int launch_residual(lbm_mix* h, long k) {
  lbm_residual_kernel<<<1, 1024, 0, h->stream>>>(h->cs[h->cur], h->cs_snap, 4L * h->L.Nx,
                                                 (double)k, h->have_snap ? 1 : 0, h->resid);
  CK(cudaGetLastError());
  h->have_snap = true;
  CK(cudaMemcpyAsync(h->h_pinned, h->resid, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return LBM_OK;
}

// Node-to-CTA schedule: rows per CTA (a multiple of TY); the per-row-block
// partials grow when a schedule needs more row blocks than allocated.
int set_rows_per_block(lbm_mix* h, int rows) {
  const int nmax = (h->L.N + TY - 1) / TY * TY;
  if (rows <= 0) rows = default_rows(h->L.N);
  if (rows % TY != 0) return set_err(LBM_EINVAL, "rows per block must be a multiple of %d", TY);
  if (rows > nmax) rows = nmax;
  const int R = (h->L.N + rows - 1) / rows;
  if (R > h->R_alloc) {
    double* cp = nullptr;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMalloc((void**)&cp, sizeof(double) * 4 * (size_t)h->L.Nx * (size_t)R));
    cudaFree(h->colpart);
    h->colpart = cp;
    h->R_alloc = R;
  }
  h->rows_per_block = rows;
  h->R = R;
  return LBM_OK;
}

int reset_diag(lbm_mix* h) {
  CK(cudaMemsetAsync(h->diag_count, 0, sizeof(unsigned long long), h->stream));
  CK(cudaMemsetAsync(h->diag, 0, sizeof(double) * DIAG_CAP * NREC, h->stream));
  h->have_snap = false;
  return LBM_OK;
}

// FP32 storage takes r and tau_q from lbm_walls_kernel when the step's grid
// holds at least WALL_KERNEL_WAVES waves of resident CTAs (3 per SM): there
// the CTA prologue's barrier costs more than a launch of its own (0.400
// against 0.406 ms on the 32768 x 512 channel).  A grid of a wave or less,
// like the channels of a parametric sweep, keeps the prologue, which costs
// less than the extra launch.  16-bit storage always uses the wall kernel.
constexpr long WALL_KERNEL_WAVES = 2;
bool uses_wall_kernel(const lbm_mix* h) {
  const long ctas = (long)h->nblocks * (long)h->R;
  return ctas >= WALL_KERNEL_WAVES * 3L * (long)(h->nsm > 0 ? h->nsm : 1);
}

int launch_step(lbm_mix* h, bool diag) {
  const int b = h->cur;
  int st = with_storage(h, [&](auto tag) -> int {
    using ST = decltype(tag);
    StepArgs<ST> a;
    a.fin = (const ST*)h->buf[b];
    a.fout = (ST*)h->buf[1 - b];
    a.refrho = h->refrho;
    a.cs_in = h->cs[b];
    a.cs_out = h->cs[1 - b];
    a.alpha = h->alpha;
    a.partials = h->partials;
    a.counter = h->counter;
    a.diag = h->diag;
    a.diag_count = h->diag_count;
    a.clprof = h->clprof;
    a.colpart = h->colpart;
    a.strip_cnt = h->strip_cnt;
    a.rows_per_block = h->rows_per_block;
    // stochastic rounding of 16-bit stores: a fresh seed every step (never 0)
    a.seed = (sizeof(ST) < 4 && h->p.rounding == LBM_ROUND_STOCHASTIC)
                 ? (host_hash32((unsigned)(h->steps + 1)) | 1u)
                 : 0u;
    a.wall_r = h->wall_r;
    a.wall_omq = h->wall_omq;
    a.pdl_early = h->pdl_early ? 1 : 0;
    // Both kernels are launched with programmatic stream serialisation, so
    // that each one's launch and CTA ramp overlap the end of the kernel
    // before it (see pdl_wait).
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.stream = h->stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool wk = sizeof(ST) < 4 || uses_wall_kernel(h);
    if (wk) {
      cfg.gridDim = dim3((h->L.Nx + 127) / 128, 4);
      cfg.blockDim = dim3(128);
      CK(cudaLaunchKernelEx(&cfg, lbm_walls_kernel<ST>, h->L, a.fin, (const float*)h->refrho,
                            (const double*)a.cs_in, (const float*)h->alpha, h->wall_r,
                            h->wall_omq));
    }
    cfg.gridDim = dim3(h->nblocks, h->R);
    cfg.blockDim = dim3(TX, TY);
    if (sizeof(ST) < 4 || !wk) {
      if (diag)
        CK(cudaLaunchKernelEx(&cfg, lbm_step_kernel<ST, true>, h->L, a));
      else
        CK(cudaLaunchKernelEx(&cfg, lbm_step_kernel<ST, false>, h->L, a));
    } else {
      if (diag)
        CK(cudaLaunchKernelEx(&cfg, lbm_step_kernel<ST, true, true>, h->L, a));
      else
        CK(cudaLaunchKernelEx(&cfg, lbm_step_kernel<ST, false, true>, h->L, a));
    }
    return LBM_OK;
  });
  if (st) return st;
  h->cur = 1 - b;
  h->steps++;
  return LBM_OK;
}

int launch_moments(lbm_mix* h, double* d_out) {
  // The state of step n is the stream of buffer P_{n-1}; right after init or
  // an upload only the buffer itself exists.
  const bool direct = (h->steps == 0);
  const int b = direct ? h->cur : 1 - h->cur;
  dim3 blk(TX, TY), grd(h->nblocks);
  int st = with_storage(h, [&](auto tag) -> int {
    using ST = decltype(tag);
    lbm_moments_kernel<ST><<<grd, blk, 0, h->stream>>>(h->L, (const ST*)h->buf[b], h->refrho,
                                                       h->cs[b], h->alpha, direct ? 1 : 0, d_out);
    CK(cudaGetLastError());
    return LBM_OK;
  });
  if (st) return st;
  if (!h->L.x_periodic) {
    lbm_moments_ends_kernel<<<2, 256, 0, h->stream>>>(h->L, d_out);
    CK(cudaGetLastError());
  }
  return LBM_OK;
}

int check_handle(const lbm_mix* h) {
  if (!h) return set_err(LBM_EINVAL, "handle is NULL");
  return LBM_OK;
}

// Latest diagnostic record (host copy). Returns LBM_ENONFINITE on NaN/Inf.
int latest_record(lbm_mix* h, double rec[NREC]) {
  unsigned long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, h->diag_count, sizeof cnt, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (cnt == 0) return set_err(LBM_EINVAL, "no step taken yet");
  CK(cudaMemcpyAsync(rec, h->diag + ((cnt - 1) % DIAG_CAP) * NREC, sizeof(double) * NREC,
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 1; k < NREC; ++k)
    if (!isfinite(rec[k])) return set_err(LBM_ENONFINITE, "non-finite diagnostic at step %llu", cnt);
  return LBM_OK;
}

}  // namespace

// ---------------------------------------------- allocation-free stepping
// Scratch of lbm_mix_step_noalloc: the per-strip partial sums, the per-strip
// and grid arrival tickets and the record counter of lbm_step_kernel, in one
// static device array so that a caller who cannot allocate device memory can
// still run a step.  Every GPU that loads the library holds it until exit:
//   partials  NOALLOC_MAX_STRIPS * NPART doubles   (64 KiB)
//   counters  NOALLOC_MAX_STRIPS + 4 words          (4 KiB + 16 B)
constexpr int NOALLOC_MAX_STRIPS = 1024;  // N_x <= 32 * 1024 = 32768 columns
constexpr size_t NOALLOC_PART_DOUBLES = (size_t)NOALLOC_MAX_STRIPS * NPART;
constexpr size_t NOALLOC_CNT_WORDS = NOALLOC_MAX_STRIPS + 4;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_PART_DOUBLES + (NOALLOC_CNT_WORDS + 1) / 2;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// The calling thread's current CUDA context (the driver's cuCtxGetCurrent,
// reached through the runtime so that the library needs no link against
// the driver library); nullptr if none is current or the query fails.
void* current_context() {
  typedef int (*CtxGetCurrent)(void**);
  static CtxGetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return (CtxGetCurrent)f;
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

// Device address of g_noalloc_scratch in the current device's context.  In
// host code the symbol's name only stands for the device array; kernels
// must be given this address.  It is looked up on the first call on a
// device and again whenever the current context is not the one it was
// looked up in (a device reset or another primary context loads the module
// anew, at another address).
int noalloc_scratch_address(double** out) {
  static std::mutex mu;
  static double* addr[64] = {};
  static void* ctx_of[64] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return set_err(LBM_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  void* ctx = current_context();
  if (!addr[dev] || !ctx || ctx != ctx_of[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return set_err(LBM_ECUDA, "cudaGetSymbolAddress(scratch) failed on device %d: %s", dev,
                     cudaGetErrorString(e));
    addr[dev] = (double*)ptr;
    ctx_of[dev] = current_context();  // the lookup made the primary context current
  }
  *out = addr[dev];
  return LBM_OK;
}

template <typename T>
int get_post_state_t(lbm_mix* h, T* f, long n) {
  int st = check_handle(h);
  if (st) return st;
  const long need = 18L * h->L.N * h->L.Nx;
  if (!f || n != need) return set_err(LBM_EINVAL, "need %ld populations", need);
  const size_t bytes = sizeof(T) * (size_t)need;
  // staging area sized for the FP64 variant, shared by both getters
  if (!h->scratch) CK(cudaMalloc((void**)&h->scratch, sizeof(double) * (size_t)need));
  dim3 blk(128), grd((h->L.Nx + 127) / 128, h->L.N, 2);
  if ((st = with_storage(h, [&](auto tag) -> int {
         using ST = decltype(tag);
         lbm_convert_kernel<ST, T><<<grd, blk, 0, h->stream>>>(h->L, (ST*)h->buf[h->cur],
                                                               h->refrho, 0, nullptr,
                                                               (T*)h->scratch);
         CK(cudaGetLastError());
         return LBM_OK;
       })))
    return st;
  CK(cudaMemcpyAsync(f, h->scratch, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

extern "C" {

void lbm_mix_default_params(lbm_mix_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->m_a = 4.003;
  p->m_b = 39.948;
  p->C_l = 0.5;
  p->C_l_out = -1.0;
  p->theta = 2.0;
  p->Kn_out = 0.1;
  p->N = 16;
  p->N_x = 0;
  p->L_over_H = 20.0;
  p->accommodation = 1.0;
  p->c_m0 = 1.016;
  p->tau_rho = 1.0;
  p->tau_e = 1.1;
  p->tau_eps = 1.2;
  p->mu_ratio_a = 1.0;
  p->mu_ratio_b = 1.0;
  p->storage = LBM_FP32;
  p->x_periodic = 0;
  p->diag_every = 1;
  p->reref_every = -1;
  p->rounding = LBM_ROUND_STOCHASTIC;
  p->wall = LBM_WALL_DBB;
}

const char* lbm_mix_strerror(int s) {
  switch (s) {
    case LBM_OK: return "success";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ENONFINITE: return "non-finite value in the state";
    case LBM_ENOTCONVERGED: return "not converged within max_steps";
    case LBM_ETIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* lbm_mix_last_error(void) { return g_err; }

void lbm_mix_destroy(lbm_mix* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->buf[0]);
  cudaFree(h->buf[1]);
  cudaFree(h->refrho);
  cudaFree(h->refrho_alt);
  cudaFree(h->cs_tmp);
  cudaFree(h->scratch);
  cudaFree(h->cs[0]);
  cudaFree(h->cs[1]);
  cudaFree(h->cs_snap);
  cudaFree(h->alpha);
  cudaFree(h->partials);
  cudaFree(h->counter);
  cudaFree(h->diag);
  cudaFree(h->diag_count);
  cudaFree(h->clprof);
  cudaFree(h->wall_r);
  cudaFree(h->wall_omq);
  cudaFree(h->colpart);
  cudaFree(h->strip_cnt);
  cudaFree(h->resid);
  cudaFree(h->mom);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaSetDevice(prev);
  delete h;
}

int lbm_mix_create(const lbm_mix_params* p, void* stream, lbm_mix** out) {
  if (!out) return set_err(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  int Nx = 0;
  int st = validate(p, &Nx);
  if (st != LBM_OK) return st;
  lbm_mix* h = new (std::nothrow) lbm_mix;
  if (!h) return set_err(LBM_ENOMEM, "host allocation failed");
  memset(h, 0, sizeof *h);
  h->p = *p;
  h->L = derive(p, Nx);
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    delete h;
    return set_err(LBM_ECUDA, "no CUDA device");
  }
  h->nblocks = (Nx + TX - 1) / TX;
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return set_err(LBM_ECUDA, "cudaStreamCreate failed");
    }
    h->own_stream = true;
  }
  h->elem = (p->storage == LBM_FP32) ? sizeof(float) : 2;
  const size_t fbytes = h->elem * 18 * (size_t)h->L.N * h->L.pitch;
  const size_t cbytes = sizeof(double) * 4 * (size_t)Nx;
  cudaError_t e = cudaSuccess;
#define ALLOC(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes))
  ALLOC(h->buf[0], fbytes);
  ALLOC(h->buf[1], fbytes);
  ALLOC(h->refrho, sizeof(float) * 2 * (size_t)Nx);
  ALLOC(h->refrho_alt, sizeof(float) * 2 * (size_t)Nx);
  ALLOC(h->cs_tmp, cbytes);
  ALLOC(h->cs[0], cbytes);
  ALLOC(h->cs[1], cbytes);
  ALLOC(h->cs_snap, cbytes);
  ALLOC(h->alpha, sizeof(float) * 2 * (size_t)Nx);
  ALLOC(h->partials, sizeof(double) * NPART * (size_t)h->nblocks);
  ALLOC(h->counter, sizeof(unsigned));
  ALLOC(h->diag, sizeof(double) * DIAG_CAP * NREC);
  ALLOC(h->diag_count, sizeof(unsigned long long));
  ALLOC(h->clprof, sizeof(double) * (size_t)Nx);
  ALLOC(h->wall_r, sizeof(float2) * 2 * (size_t)Nx);
  ALLOC(h->wall_omq, sizeof(float) * 2 * (size_t)Nx);
  // Row blocks: split each strip's rows over R CTAs of DEFAULT_ROWS rows so
  // that the grid holds many waves of CTAs on the device's SMs and its last,
  // partial wave is a small share of the launch.
  h->rows_per_block = default_rows(h->L.N);
  h->R = (h->L.N + h->rows_per_block - 1) / h->rows_per_block;
  h->R_alloc = h->R;
  ALLOC(h->colpart, sizeof(double) * 4 * (size_t)Nx * (size_t)h->R);
  ALLOC(h->strip_cnt, sizeof(unsigned) * (size_t)h->nblocks);
  ALLOC(h->resid, sizeof(double));
#undef ALLOC
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_pinned, sizeof(double) * 64);
  if (e != cudaSuccess) {
    int code = (e == cudaErrorMemoryAllocation) ? LBM_ENOMEM : LBM_ECUDA;
    set_err(code, "allocation failed: %s", cudaGetErrorString(e));
    cudaGetLastError();
    lbm_mix_destroy(h);
    return code;
  }
  // zero everything so that padding and ghost columns hold defined values
  e = cudaMemsetAsync(h->buf[0], 0, fbytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->buf[1], 0, fbytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->counter, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(h->strip_cnt, 0, sizeof(unsigned) * (size_t)h->nblocks, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->cs[0], 0, cbytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->cs[1], 0, cbytes, h->stream);
  if (e == cudaSuccess) {
    float* a = (float*)malloc(sizeof(float) * 4 * Nx);
    if (!a) e = cudaErrorMemoryAllocation;
    else {
      for (int k = 0; k < 2 * Nx; ++k) a[k] = (float)p->accommodation;
      // reference densities: the initial profile of lbm_mix_init
      float* rb = a + 2 * Nx;
      for (int x = 0; x < Nx; ++x) {
        double t = h->L.x_periodic ? 1.0 : (double)x / (Nx - 1);
        double n = h->L.x_periodic ? 1.0 : p->theta + (1.0 - p->theta) * t;
        double Cl = h->L.C_in + (h->L.C_out - h->L.C_in) * t;
        for (int sp = 0; sp < 2; ++sp) {
          double C = (sp == h->L.light) ? Cl : 1.0 - Cl;
          rb[sp * Nx + x] = (float)(n * C * h->L.mh[sp]);
        }
      }
      e = cudaMemcpyAsync(h->alpha, a, sizeof(float) * 2 * Nx, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->refrho, rb, sizeof(float) * 2 * Nx, cudaMemcpyHostToDevice,
                            h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      free(a);
    }
  }
  if (e != cudaSuccess) {
    set_err(LBM_ECUDA, "initialisation failed: %s", cudaGetErrorString(e));
    lbm_mix_destroy(h);
    return LBM_ECUDA;
  }
  if (reset_diag(h) != LBM_OK) {
    lbm_mix_destroy(h);
    return LBM_ECUDA;
  }
  *out = h;
  return LBM_OK;
}

int lbm_mix_init(lbm_mix* h) {
  int st = check_handle(h);
  if (st) return st;
  h->cur = 0;
  h->steps = 0;
  // the initial state is the rest equilibrium of the reference densities:
  // all stored deviations are zero
  CK(cudaMemsetAsync(h->buf[0], 0, h->elem * 18 * (size_t)h->L.N * h->L.pitch,
                     h->stream));
  if ((st = launch_colsum(h, 0))) return st;
  return reset_diag(h);
}

int lbm_mix_step(lbm_mix* h, long nsteps) {
  int st = check_handle(h);
  if (st) return st;
  if (nsteps < 0) return set_err(LBM_EINVAL, "nsteps < 0");
  const long reref = h->p.reref_every >= 0 ? h->p.reref_every
                                           : (h->p.storage == LBM_FP32 ? 0 : 256);
  // diagnostics on every diag_every-th step and on the last step of the call
  for (long t = 0; t < nsteps; ++t) {
    const bool diag = (t == nsteps - 1) || ((h->steps + 1) % h->p.diag_every == 0);
    if ((st = launch_step(h, diag))) return st;
    if (reref > 0 && h->steps % reref == 0 && (st = rereference(h))) return st;
  }
  return LBM_OK;
}

int lbm_mix_rereference(lbm_mix* h) {
  int st = check_handle(h);
  if (st) return st;
  return rereference(h);
}

int lbm_mix_run_to_steady(lbm_mix* h, double tol, long max_steps, long check_every,
                          long* steps_out, double* residual_out) {
  int st = check_handle(h);
  if (st) return st;
  if (!(tol > 0) || max_steps < 0 || check_every < 1)
    return set_err(LBM_EINVAL, "need tol > 0, max_steps >= 0, check_every >= 1");
  long taken = 0;
  double R = INFINITY;
  int result = LBM_ENOTCONVERGED;
  while (taken < max_steps) {
    long k = check_every < max_steps - taken ? check_every : max_steps - taken;
    if ((st = lbm_mix_step(h, k))) return st;
    taken += k;
    if ((st = launch_residual(h, k))) return st;
    CK(cudaStreamSynchronize(h->stream));
    R = h->h_pinned[0];
    if (isnan(R)) {
      result = set_err(LBM_ENONFINITE, "non-finite residual after %ld steps", taken);
      break;
    }
    if (R <= tol) {
      result = LBM_OK;
      break;
    }
  }
  if (steps_out) *steps_out = taken;
  if (residual_out) *residual_out = R;
  if (result == LBM_ENOTCONVERGED)
    set_err(LBM_ENOTCONVERGED, "residual %.3e above %.3e after %ld steps", R, tol, taken);
  return result;
}

int lbm_mix_set_rows_per_block(lbm_mix* h, int rows) {
  int st = check_handle(h);
  if (st) return st;
  return set_rows_per_block(h, rows);
}

int lbm_mix_tune_rows(lbm_mix* h, const int* candidates, int n, long steps, int* best_rows) {
  int st = check_handle(h);
  if (st) return st;
  static const int kDefault[] = {64, 72, 80, 88, 96, 112, 128};
  if (!candidates) {
    candidates = kDefault;
    n = (int)(sizeof kDefault / sizeof kDefault[0]);
  }
  if (n < 1 || steps < 1) return set_err(LBM_EINVAL, "need n >= 1 candidates and steps >= 1");
  for (int k = 0; k < n; ++k)
    if (candidates[k] <= 0 || candidates[k] % TY != 0)
      return set_err(LBM_EINVAL, "candidate %d: rows must be a positive multiple of %d", k, TY);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_err(LBM_ECUDA, "cudaEventCreate failed");
  }
  int best = h->rows_per_block;
  float best_ms = INFINITY;
  for (int k = 0; k < n && st == LBM_OK; ++k) {
    if ((st = set_rows_per_block(h, candidates[k]))) break;
    // two untimed steps settle the new schedule (first-touch of its buffers)
    if ((st = lbm_mix_step(h, 2))) break;
    if (cudaEventRecord(e0, h->stream) != cudaSuccess ||
        (st = lbm_mix_step(h, steps)) != LBM_OK || cudaEventRecord(e1, h->stream) != cudaSuccess ||
        cudaEventSynchronize(e1) != cudaSuccess) {
      if (st == LBM_OK) st = set_err(LBM_ECUDA, "timing a candidate schedule failed");
      break;
    }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = h->rows_per_block;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  if ((st = set_rows_per_block(h, best))) return st;
  if (best_rows) *best_rows = best;
  return LBM_OK;
}

int lbm_mix_moments_device(lbm_mix* h, double* d_out) {
  int st = check_handle(h);
  if (st) return st;
  if (!d_out) return set_err(LBM_EINVAL, "d_out is NULL");
  return launch_moments(h, d_out);
}

int lbm_mix_moments(lbm_mix* h, double* rho_a, double* rho_b, double* ua_x, double* ua_y,
                    double* ub_x, double* ub_y) {
  int st = check_handle(h);
  if (st) return st;
  const size_t plane = (size_t)h->L.N * h->L.Nx;
  if (!h->mom) CK(cudaMalloc((void**)&h->mom, sizeof(double) * 6 * plane));
  if ((st = launch_moments(h, h->mom))) return st;
  double* outs[6] = {rho_a, rho_b, ua_x, ua_y, ub_x, ub_y};
  for (int k = 0; k < 6; ++k)
    if (outs[k])
      CK(cudaMemcpyAsync(outs[k], h->mom + k * plane, sizeof(double) * plane,
                         cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mix_device_ptrs(lbm_mix* h, void** populations, long* n_populations, void** refrho,
                        void** alpha, void** colsum) {
  int st = check_handle(h);
  if (st) return st;
  if (populations) *populations = h->buf[h->cur];
  if (n_populations) *n_populations = 18L * h->L.N * h->L.pitch;
  if (refrho) *refrho = h->refrho;
  if (alpha) *alpha = h->alpha;
  if (colsum) *colsum = h->cs[h->cur];
  return LBM_OK;
}

int lbm_mix_volume_flow(lbm_mix* h, int x, double* Qv) {
  int st = check_handle(h);
  if (st) return st;
  if (!Qv) return set_err(LBM_EINVAL, "Qv is NULL");
  if (x < 0) x = h->L.x_periodic ? 0 : h->L.Nx - 2;
  if (x >= h->L.Nx || (!h->L.x_periodic && (x < 1 || x > h->L.Nx - 2)))
    return set_err(LBM_EINVAL, "column %d is not an updated column", x);
  const size_t plane = (size_t)h->L.N * h->L.Nx;
  if (!h->mom) CK(cudaMalloc((void**)&h->mom, sizeof(double) * 6 * plane));
  if ((st = launch_moments(h, h->mom))) return st;
  lbm_volume_flow_kernel<<<1, 256, 0, h->stream>>>(h->mom, h->L.N, h->L.Nx, x, h->resid);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(h->h_pinned, h->resid, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *Qv = h->h_pinned[0];
  if (!isfinite(*Qv)) return set_err(LBM_ENONFINITE, "non-finite volume flow");
  return LBM_OK;
}

int lbm_mix_separation(lbm_mix* h, double* CL, double* Cl_tilde, double* mdot_a, double* mdot_b,
                       double* Cl_profile, int* x_min) {
  int st = check_handle(h);
  if (st) return st;
  double rec[NREC];
  if ((st = latest_record(h, rec))) return st;
  if (CL) *CL = rec[1];
  if (Cl_tilde) *Cl_tilde = rec[2];
  if (mdot_a) *mdot_a = rec[3];
  if (mdot_b) *mdot_b = rec[4];
  if (x_min) *x_min = (int)rec[5];
  if (Cl_profile) {
    CK(cudaMemcpyAsync(Cl_profile, h->clprof, sizeof(double) * h->L.Nx, cudaMemcpyDeviceToHost,
                       h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return LBM_OK;
}

int lbm_mix_history(lbm_mix* h, double* rec, long max_records, long* count) {
  int st = check_handle(h);
  if (st) return st;
  if (!rec || max_records < 0 || !count) return set_err(LBM_EINVAL, "bad history arguments");
  unsigned long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, h->diag_count, sizeof cnt, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  long have = (long)(cnt < (unsigned long long)DIAG_CAP ? cnt : DIAG_CAP);
  long take = have < max_records ? have : max_records;
  for (long k = 0; k < take; ++k) {
    unsigned long long idx = (cnt - take + k) % DIAG_CAP;
    CK(cudaMemcpyAsync(rec + k * NREC, h->diag + idx * NREC, sizeof(double) * NREC,
                       cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  *count = take;
  return LBM_OK;
}

int lbm_mix_set_accommodation_field(lbm_mix* h, const double* alpha, long n) {
  int st = check_handle(h);
  if (st) return st;
  if (!alpha || n != 2L * h->L.Nx) return set_err(LBM_EINVAL, "need 2*N_x accommodation values");
  float* a = (float*)malloc(sizeof(float) * n);
  if (!a) return set_err(LBM_ENOMEM, "host allocation failed");
  for (long k = 0; k < n; ++k) {
    if (!(alpha[k] > 0 && alpha[k] <= 1)) {
      free(a);
      return set_err(LBM_EINVAL, "accommodation[%ld] = %g outside (0,1]", k, alpha[k]);
    }
    a[k] = (float)alpha[k];
  }
  cudaError_t e = cudaMemcpyAsync(h->alpha, a, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  free(a);
  if (e != cudaSuccess) return set_err(LBM_ECUDA, "upload failed: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_mix_set_post_state(lbm_mix* h, const float* f, long n) {
  int st = check_handle(h);
  if (st) return st;
  const long need = 18L * h->L.N * h->L.Nx;
  if (!f || n != need) return set_err(LBM_EINVAL, "need %ld populations", need);
  h->cur = 0;
  h->steps = 0;
  if (!h->scratch) CK(cudaMalloc((void**)&h->scratch, sizeof(double) * (size_t)need));
  CK(cudaMemcpyAsync(h->scratch, f, sizeof(float) * (size_t)need, cudaMemcpyHostToDevice,
                     h->stream));
  {
    dim3 blk(128), grd((h->L.Nx + 127) / 128, h->L.N, 2);
    if ((st = with_storage(h, [&](auto tag) -> int {
           using ST = decltype(tag);
           lbm_convert_kernel<ST, float><<<grd, blk, 0, h->stream>>>(
               h->L, (ST*)h->buf[0], h->refrho, 1, (const float*)h->scratch, (float*)nullptr);
           CK(cudaGetLastError());
           return LBM_OK;
         })))
      return st;
  }
  if ((st = launch_colsum(h, 0))) return st;
  if ((st = reset_diag(h))) return st;
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mix_get_post_state(lbm_mix* h, float* f, long n) { return get_post_state_t(h, f, n); }

int lbm_mix_get_post_state_f64(lbm_mix* h, double* f, long n) {
  return get_post_state_t(h, f, n);
}

int lbm_mix_dims(const lbm_mix* h, int* N, int* N_x, long* steps) {
  int st = check_handle(h);
  if (st) return st;
  if (N) *N = h->L.N;
  if (N_x) *N_x = h->L.Nx;
  if (steps) *steps = h->steps;
  return LBM_OK;
}

int lbm_mix_launches_per_step(const lbm_mix* h) {
  int st = check_handle(h);
  if (st) return st;
  return (h->elem < 4 || uses_wall_kernel(h)) ? 2 : 1;
}

int lbm_mix_sync(lbm_mix* h) {
  int st = check_handle(h);
  if (st) return st;
  CK(cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

int lbm_mix_eval_special(const double* x, double* e1, double* psi, long n) {
  if (!x || n < 0) return set_err(LBM_EINVAL, "bad arguments");
  if (n == 0) return LBM_OK;
  for (long k = 0; k < n; ++k)
    if (!(x[k] > 0)) return set_err(LBM_EINVAL, "x[%ld] must be > 0", k);
  double *dx = nullptr, *de = nullptr, *dp = nullptr;
  const size_t b = sizeof(double) * n;
  cudaError_t e = cudaMalloc((void**)&dx, b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&de, b);
  if (e == cudaSuccess) e = cudaMalloc((void**)&dp, b);
  if (e == cudaSuccess) e = cudaMemcpy(dx, x, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    lbm_special_kernel<<<(unsigned)((n + 255) / 256), 256>>>(dx, de, dp, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && e1) e = cudaMemcpy(e1, de, b, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && psi) e = cudaMemcpy(psi, dp, b, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(de);
  cudaFree(dp);
  if (e != cudaSuccess) return set_err(LBM_ECUDA, "eval_special: %s", cudaGetErrorString(e));
  return LBM_OK;
}

int lbm_mix_step_noalloc(const lbm_mix_params* p, const float* d_in, float* d_out,
                         const float* d_refrho, const float* d_alpha, const double* d_colsum_in,
                         double* d_colsum_out, double* d_record, double* d_cl_profile,
                         void* stream) {
  int Nx = 0;
  int st = validate(p, &Nx);
  if (st != LBM_OK) return st;
  if (!d_in || !d_out || !d_refrho || !d_alpha || !d_colsum_in || !d_colsum_out || !d_record ||
      !d_cl_profile)
    return set_err(LBM_EINVAL, "lbm_mix_step_noalloc: every buffer must be a device pointer");
  if (d_in == d_out) return set_err(LBM_EINVAL, "lbm_mix_step_noalloc: d_in and d_out alias");
  if (p->storage != LBM_FP32)
    return set_err(LBM_EINVAL, "lbm_mix_step_noalloc: FP32 storage only");
  const int nstrips = (Nx + TX - 1) / TX;
  if (nstrips > NOALLOC_MAX_STRIPS)
    return set_err(LBM_EINVAL,
                   "lbm_mix_step_noalloc: N_x = %d exceeds the %d columns its static scratch "
                   "covers",
                   Nx, NOALLOC_MAX_STRIPS * TX);
  double* scratch = nullptr;
  if ((st = noalloc_scratch_address(&scratch))) return st;
  const Lat L = derive(p, Nx);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* cnt = (unsigned*)(scratch + NOALLOC_PART_DOUBLES);
  // tickets and the record counter must start at zero; the partials are
  // overwritten before they are read
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned) * NOALLOC_CNT_WORDS, s));
  StepArgs<float> a;
  a.fin = d_in;
  a.fout = d_out;
  a.refrho = d_refrho;
  a.cs_in = d_colsum_in;
  a.cs_out = d_colsum_out;
  a.alpha = d_alpha;
  a.partials = scratch;
  a.strip_cnt = cnt;
  a.counter = cnt + NOALLOC_MAX_STRIPS;
  a.diag_count = (unsigned long long*)(cnt + NOALLOC_MAX_STRIPS + 2);
  a.diag = d_record;  // the zeroed counter puts the record at index 0
  a.clprof = d_cl_profile;
  a.colpart = nullptr;  // one row block per strip: no row-block partials
  a.rows_per_block = (L.N + TY - 1) / TY * TY;
  a.seed = 0u;  // FP32 storage: no rounding to 16 bits
  a.wall_r = nullptr;  // FP32 storage: the wall prologue computes r and tau_q
  a.wall_omq = nullptr;
  a.pdl_early = 0;  // a plain launch: the trigger would be a no-op
  dim3 blk(TX, TY), grd(nstrips, 1);
  lbm_step_kernel<float, true><<<grd, blk, 0, s>>>(L, a);
  CK(cudaGetLastError());
  return LBM_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- sweeps
// A parametric study (Table 1) runs many independent channels.  Each
// instance keeps its own handle and stream; K steps of an instance are
// captured once as a CUDA graph (K fused step launches) and replayed, so the
// host issues one graph launch per instance per convergence check and the
// instances' kernels run concurrently, filling the GPU with channels that
// are each too small to fill it alone.  The first blocks of
// lbm_sweep_run_to_steady can serve as an autotuner of the node-to-CTA
// schedule (rows per CTA): each candidate schedule runs one real block of
// steps, the fastest is kept.  Schedules change only the order of the FP64
// column reductions, not the time integration.
// What a captured graph has baked into its launches besides the handle's
// fixed buffers: the buffer parity it starts from, the schedule (rows per
// CTA, row blocks and their partials), the reference-density table (swapped
// by re-referencing) and the step phase that decides which captured steps
// reduce diagnostics.  A graph is replayed only while all of them match.
struct SweepCapKey {
  int cur, rows, R;
  const void* colpart;
  const void* refrho;
  long phase;
};

struct lbm_sweep {
  int n = 0;
  lbm_mix** h = nullptr;
  cudaGraphExec_t* exec = nullptr;
  long* exec_K = nullptr;  // steps captured in exec[i]; 0 = none
  SweepCapKey* key = nullptr;  // state each graph was captured from
  int policy = -1;         // schedule in use (-1: the library default)
  double round_ms[LBM_SWEEP_NPOLICY] = {};
};

namespace {

SweepCapKey cap_key(const lbm_mix* h) {
  return SweepCapKey{h->cur, h->rows_per_block, h->R, h->colpart, h->refrho,
                     h->steps % h->p.diag_every};
}

bool same_key(const SweepCapKey& a, const SweepCapKey& b) {
  return a.cur == b.cur && a.rows == b.rows && a.R == b.R && a.colpart == b.colpart &&
         a.refrho == b.refrho && a.phase == b.phase;
}

// Instance i has a graph of K steps that is valid for its current state.
bool graph_valid(const lbm_sweep* s, int i, long K) {
  return s->exec[i] && s->exec_K[i] == K && same_key(s->key[i], cap_key(s->h[i]));
}

// Rows per CTA of instance h under schedule policy p.
int policy_rows(const lbm_mix* h, int p) {
  const int N = h->L.N;
  switch (p) {
    case 0: return 0;  // library default: row blocks of DEFAULT_ROWS rows
    case 1: return 64;
    case 2: return 32;
    case 3: return 16;
    default: {  // fill: about two CTAs per SM for this instance alone
      const long want = 2L * (h->nsm > 0 ? h->nsm : 1);
      long rows = ((long)N * h->nblocks + want - 1) / want;
      rows = (rows + TY - 1) / TY * TY;
      if (rows < 16) rows = 16;
      if (rows > 128) rows = 128;
      return (int)rows;
    }
  }
}

void drop_graph(lbm_sweep* s, int i) {
  if (s->exec[i]) cudaGraphExecDestroy(s->exec[i]);
  s->exec[i] = nullptr;
  s->exec_K[i] = 0;
}

// K (even) steps of instance i as one graph executable.  Capturing records
// the launches without running them, so the host-side step count and buffer
// parity are restored afterwards.
int capture_steps(lbm_sweep* s, int i, long K) {
  lbm_mix* h = s->h[i];
  drop_graph(s, i);
  const long steps0 = h->steps;
  const int cur0 = h->cur;
  const SweepCapKey key = cap_key(h);
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int st = lbm_mix_step(h, K);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  h->steps = steps0;
  h->cur = cur0;
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess)
    return set_err(LBM_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&s->exec[i], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    s->exec[i] = nullptr;
    return set_err(LBM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  s->exec_K[i] = K;
  s->key[i] = key;
  return LBM_OK;
}

int apply_policy(lbm_sweep* s, int p) {
  for (int i = 0; i < s->n; ++i) {
    lbm_mix* h = s->h[i];
    const int before = h->rows_per_block;
    int st = set_rows_per_block(h, policy_rows(h, p));
    if (st) return st;
    if (h->rows_per_block != before) drop_graph(s, i);
  }
  s->policy = p;
  return LBM_OK;
}

double now_ms() {
  struct timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return ts.tv_sec * 1e3 + ts.tv_nsec * 1e-6;
}

}  // namespace

extern "C" {

int lbm_sweep_create(const lbm_mix_params* params, int n, lbm_sweep** out) {
  if (!out) return set_err(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  if (!params || n < 1) return set_err(LBM_EINVAL, "need n >= 1 parameter sets");
  for (int i = 0; i < n; ++i) {
    int Nx = 0;
    int st = validate(&params[i], &Nx);
    if (st) {
      char why[sizeof g_err];
      memcpy(why, g_err, sizeof why);
      return set_err(st, "instance %d: %s", i, why);
    }
    if (params[i].storage != LBM_FP32)
      return set_err(LBM_EINVAL, "instance %d: sweeps run FP32 storage only", i);
  }
  lbm_sweep* s = new (std::nothrow) lbm_sweep;
  if (!s) return set_err(LBM_ENOMEM, "host allocation failed");
  s->h = (lbm_mix**)calloc(n, sizeof(lbm_mix*));
  s->exec = (cudaGraphExec_t*)calloc(n, sizeof(cudaGraphExec_t));
  s->exec_K = (long*)calloc(n, sizeof(long));
  s->key = (SweepCapKey*)calloc(n, sizeof(SweepCapKey));
  if (!s->h || !s->exec || !s->exec_K || !s->key) {
    lbm_sweep_destroy(s);
    return set_err(LBM_ENOMEM, "host allocation failed");
  }
  s->n = n;
  for (int i = 0; i < n; ++i) {
    lbm_mix_params p = params[i];
    p.reref_every = 0;
    int st = lbm_mix_create(&p, nullptr, &s->h[i]);  // own stream per instance
    if (st) {
      lbm_sweep_destroy(s);
      return st;
    }
    s->h[i]->pdl_early = true;
  }
  *out = s;
  return LBM_OK;
}

void lbm_sweep_destroy(lbm_sweep* s) {
  if (!s) return;
  for (int i = 0; i < s->n; ++i) {
    if (s->exec) drop_graph(s, i);
    if (s->h) lbm_mix_destroy(s->h[i]);
  }
  free(s->h);
  free(s->exec);
  free(s->exec_K);
  free(s->key);
  delete s;
}

int lbm_sweep_init(lbm_sweep* s) {
  if (!s) return set_err(LBM_EINVAL, "sweep is NULL");
  for (int i = 0; i < s->n; ++i) {
    int st = lbm_mix_init(s->h[i]);
    if (st) return st;
  }
  return LBM_OK;
}

int lbm_sweep_step(lbm_sweep* s, long nsteps) {
  if (!s) return set_err(LBM_EINVAL, "sweep is NULL");
  if (nsteps < 0) return set_err(LBM_EINVAL, "nsteps < 0");
  for (int i = 0; i < s->n; ++i) {
    int st = lbm_mix_step(s->h[i], nsteps);
    if (st) return st;
  }
  for (int i = 0; i < s->n; ++i) CK(cudaStreamSynchronize(s->h[i]->stream));
  return LBM_OK;
}

int lbm_sweep_run_to_steady(lbm_sweep* s, double tol, long max_steps, long check_every,
                            int autotune, long* steps_out, double* residual_out,
                            int* status_out) {
  if (!s) return set_err(LBM_EINVAL, "sweep is NULL");
  if (!(tol > 0) || max_steps < 0 || check_every < 2 || check_every % 2 != 0)
    return set_err(LBM_EINVAL, "need tol > 0, max_steps >= 0, even check_every >= 2");
  const int n = s->n;
  long* taken = (long*)calloc(n, sizeof(long));
  double* R = (double*)malloc(n * sizeof(double));
  int* status = (int*)malloc(n * sizeof(int));
  int* act = (int*)malloc(n * sizeof(int));
  if (!taken || !R || !status || !act) {
    free(taken), free(R), free(status), free(act);
    return set_err(LBM_ENOMEM, "host allocation failed");
  }
  int na = 0;
  for (int i = 0; i < n; ++i) {
    R[i] = INFINITY;
    status[i] = LBM_ENOTCONVERGED;
    // one diagnostic record per graph: the captured pattern repeats
    s->h[i]->p.diag_every = (int)check_every;
    if (max_steps > 0) act[na++] = i;
  }
  int st = LBM_OK;
  int trial = autotune ? 0 : -1;  // next schedule to try
  if (!autotune && s->policy < 0) st = apply_policy(s, 0);
  while (na > 0 && st == LBM_OK) {
    if (trial >= 0 && (st = apply_policy(s, trial))) break;
    // every active instance advances k steps: a replayed graph when k is
    // the captured length, plain launches for a shorter last block
    const long left = max_steps - taken[act[0]];
    const long k = check_every < left ? check_every : left;
    // (re)capture where no graph exists or the state moved away from the one
    // it was captured from (odd step counts, state uploads, schedule changes,
    // re-referencing through the borrowed handle)
    for (int a = 0; a < na && !st; ++a)
      if (k == check_every && !graph_valid(s, act[a], k)) st = capture_steps(s, act[a], k);
    if (st) break;
    const double t0 = now_ms();
    for (int a = 0; a < na && !st; ++a) {
      lbm_mix* h = s->h[act[a]];
      if (k == check_every) {
        cudaError_t e = cudaGraphLaunch(s->exec[act[a]], h->stream);
        if (e != cudaSuccess) st = set_err(LBM_ECUDA, "graph launch: %s", cudaGetErrorString(e));
        h->steps += k;
      } else {
        st = lbm_mix_step(h, k);
      }
      if (!st) st = launch_residual(h, k);
    }
    if (st) break;
    int nb = 0;
    for (int a = 0; a < na; ++a) {
      const int i = act[a];
      lbm_mix* h = s->h[i];
      cudaError_t e = cudaStreamSynchronize(h->stream);
      if (e != cudaSuccess) {
        st = set_err(LBM_ECUDA, "instance %d: %s", i, cudaGetErrorString(e));
        break;
      }
      taken[i] += k;
      R[i] = h->h_pinned[0];
      if (isnan(R[i])) status[i] = LBM_ENONFINITE;
      else if (R[i] <= tol) status[i] = LBM_OK;
      else if (taken[i] < max_steps) act[nb++] = i;
    }
    if (st) break;
    if (trial >= 0) {
      s->round_ms[trial] = now_ms() - t0;
      if (++trial == LBM_SWEEP_NPOLICY) {
        int best = 0;
        for (int p = 1; p < LBM_SWEEP_NPOLICY; ++p)
          if (s->round_ms[p] < s->round_ms[best]) best = p;
        trial = -1;
        st = apply_policy(s, best);
      }
    }
    na = nb;
  }
  for (int i = 0; i < n; ++i) {
    if (steps_out) steps_out[i] = taken[i];
    if (residual_out) residual_out[i] = R[i];
    if (status_out) status_out[i] = status[i];
  }
  free(taken), free(R), free(status), free(act);
  return st;
}

int lbm_sweep_instance(lbm_sweep* s, int k, lbm_mix** out) {
  if (!s || !out || k < 0 || k >= s->n) return set_err(LBM_EINVAL, "bad sweep, index or out");
  *out = s->h[k];
  return LBM_OK;
}

int lbm_sweep_schedule(lbm_sweep* s, int* policy, int* rows_per_block, double* round_ms) {
  if (!s) return set_err(LBM_EINVAL, "sweep is NULL");
  if (policy) *policy = s->policy;
  if (rows_per_block)
    for (int i = 0; i < s->n; ++i) rows_per_block[i] = s->h[i]->rows_per_block;
  if (round_ms)
    for (int p = 0; p < LBM_SWEEP_NPOLICY; ++p) round_ms[p] = s->round_ms[p];
  return LBM_OK;
}

}  // extern "C"

// ------------------------------------------- helpers for other translation units
#include "lbm_internal.h"

int lbm_internal_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int lbm_internal_validate(const lbm_mix_params* p, int* Nx_out) { return validate(p, Nx_out); }
