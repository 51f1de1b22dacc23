// lbm_adjoint.cu — FP64 forward replay and discrete adjoint of the
// two-species MRT-LBM time step (sm_103a), behind the lbm_adj_* entry points
// of include/lbm_mix.h.
//
// The forward map here is the same time step as lbm_step_kernel (Sec. 3:
// pull-streaming with the diffuse-bounce-back walls of Eqs. bot, bot2, R and
// the extrapolation-correction ends of Eqs. rho1, rho2, moments of
// Eq. rhou, effective relaxation times of Eqs. EQFrb, EQFrsp, psi, taos,
// taoq, A12, and the MRT collision of Eqs. MR, m, S, feq), written in FP64
// on the full populations in a plain [species][i][row][column] layout.  It
// is the map the adjoint differentiates, so the gradient is exact for it
// (up to FP64 rounding).
//
// One step t maps the post-collision state f^{t-1} to f^t through
//   r(x, wall)  = R(alpha, m_x of f^{t-1} at the wall node)        per column
//   kappa_s     = N rho_s,in / sum_j (2 rho_s(1, j) - rho_s(2, j)) per end
//   g           = Pull(f^{t-1}; r, kappa)                          per node
//   tau_q(x, w) = TQ(moments of g at the wall node, alpha)         per column
//   f^t         = Collide(g; tau_q of the node's half, y)          per node
// and the adjoint step runs these pieces backwards: the node-local reverse
// of Collide (hand-derived, below), the reverse of TQ into the wall nodes'
// g adjoints, the transpose of Pull as a gather over the nodes each
// population was pulled by (with the DBB and ghost-column terms), and the
// reverses of R and kappa.  Parameter adjoints: theta enters rho_in (kappa)
// and the initial state; Kn_out scales mu and with it every mean free path
// (accumulated as d/d ln mu); alpha enters R and TQ per wall node.
//
// All reductions are owned by one thread or one block in a fixed order, so
// the gradient is deterministic.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "lbm_internal.h"

#define CKA(call)                                                                       \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return lbm_internal_error(LBM_ECUDA, "%s failed: %s (%s:%d)", #call,               \
                                cudaGetErrorString(e_), __FILE__, __LINE__);            \
  } while (0)

namespace {

// Programmatic dependent launch of the per-step kernel sequences: each
// kernel lets the next one in its stream launch once all of its own CTAs
// run (launch_dependents), and waits for the previous one's completion and
// memory (wait) before its first global memory access, so that launches
// and CTA ramps overlap the end of the kernel before.  Both return at once
// for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr double kPiD = 3.14159265358979323846;
constexpr double kEulerGamma = 0.57721566490153286061;
// D2Q9 velocities c_i = (cxd(i), cyd(i)) (Eq. c).  Compile-time functions,
// not a table: in the unrolled loops the entries of M (Eq. m) and of the
// momenta fold into the code, so the zero entries cost nothing and the unit
// ones an add.
__host__ __device__ constexpr int cxd(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cyd(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// acc + c x for a coefficient c known at compile time: nothing for c = 0, an
// add or a subtraction for c = +-1, one fma otherwise (for finite x the value
// fma(c, x, acc) gives in every case; the compiler may not drop 0 x itself).
__device__ __forceinline__ double macc(double acc, double c, double x) {
  if (c == 0.0) return acc;
  if (c == 1.0) return acc + x;
  if (c == -1.0) return acc - x;
  return fma(c, x, acc);
}

// FP64 lattice constants of one problem.
struct AL {
  int N, Nx, x_periodic, light;
  double s[2], mh[2], cw[2][3];  // rest weights w_i alpha_si: rest, axis, diagonal
  double c_lam, c_xl[2], c_ts, c_td, om_e, om_eps, c_m0, H;
  double inv_c_lam, inv_c_xl[2];  // reciprocals (multiplications replace FP64 divisions)
  double rho_in[2], rho_out[2], C_in, C_out, theta;
};

// ------------------------------------------------ special functions (FP64)
// E_1 = E_i of Eq. psi in FP64, the FP64 pipe being the bound of the adjoint
// kernels (six E_1 per node per step).  0 < x <= 1: the convergent series
// (Abramowitz & Stegun 5.1.11) with a fixed number of terms (remainder
// below 1e-20) by Horner's rule; 1 < x <= 32: R(x) = x e^x E_1(x), smooth
// and between 0.59 and 0.97, as a Chebyshev series on [1,2], [2,4], [4,8],
// [8,16], [16,32] (interpolants of R fitted in 40-digit arithmetic by
// gen_e1_table.py, relative error below 2e-16), summed by Clenshaw's
// recurrence; x > 32: the continued fraction (A&S 5.1.22, modified Lentz,
// a handful of terms there).  No loop but the last has a data-dependent
// length.
// BEGIN generated E_1 tables (gen_e1_table.py)
constexpr int kE1SeriesTerms = 20;
__constant__ double kE1Series[kE1SeriesTerms] = {  // (-1)^k / (k k!), k = 1..
    -1.0,
    0.25,
    -0.055555555555555555556,
    0.010416666666666666667,
    -0.0016666666666666666667,
    0.00023148148148148148148,
    -0.000028344671201814058957,
    3.1001984126984126984e-6,
    -3.061924358220654517e-7,
    2.7557319223985890653e-8,
    -2.2774643986765198886e-9,
    1.7397297489890082483e-10,
    -1.2353110643708934307e-11,
    8.1933897126640890813e-13,
    -5.0981091545465443173e-14,
    2.9871733327421158109e-15,
    -1.6537983849091298607e-16,
    8.6773372047701258123e-18,
    -4.3266501298022787984e-19,
    2.0551588116560824292e-20};
constexpr int kE1ChebTerms = 20;
__constant__ double kE1Cheb[5][kE1ChebTerms] = {  // x e^x E_1(x) on [1,2] .. [16,32]
    {  // [1, 2], max relative error 1.5e-16
     0.66602904785893381259,
     0.062425288438637690354,
     -0.0064399715225844760029,
     0.00071881049652994166717,
     -0.000085371489910101236718,
     0.000010648380975570467222,
     -1.3809135417546289139e-6,
     1.8477934175040391861e-7,
     -2.5364639654694246794e-8,
     3.5560115645720432054e-9,
     -5.0741153091797847352e-10,
     7.3492752014463539301e-11,
     -1.078152203046921324e-11,
     1.5992380399775897593e-12,
     -2.3951298013872688691e-13,
     3.6176510021764167969e-14,
     -5.5082552205829415582e-15,
     8.6349750770716804233e-16,
     -1.2997392722785466931e-16,
     0.0},
    {  // [2, 4], max relative error 1.4e-16
     0.78023590097585564412,
     0.050579111577321273969,
     -0.0061138064664468708916,
     0.00076986586051874297637,
     -0.00010029543689856821373,
     0.000013441723236134673213,
     -1.8447925285347978064e-6,
     2.5831692135853972289e-7,
     -3.6793586219991993821e-8,
     5.318025436335566907e-9,
     -7.784409115294749227e-10,
     1.1520951705973502714e-10,
     -1.721671160265668828e-11,
     2.5948940888289542991e-12,
     -3.9407860062066585244e-13,
     6.0254449305202488572e-14,
     -9.2692537700148199283e-15,
     1.4346100679077652733e-15,
     -2.283383004897064056e-16,
     3.4804904108859155755e-17},
    {  // [4, 8], max relative error 2.0e-16
     0.86680483734339862145,
     0.035729512355926419271,
     -0.0048959245535215693208,
     0.00068348200964272786034,
     -0.000096976631812688221139,
     0.000013956364689041613815,
     -2.0337277146399378673e-6,
     2.9963382373397474592e-7,
     -4.4578239842876728156e-8,
     6.6899752178875340627e-9,
     -1.0118056680554136366e-9,
     1.5409816786636522465e-10,
     -2.3617216919622858371e-11,
     3.6402643341138812429e-12,
     -5.640079104779016553e-13,
     8.7800007595891105482e-14,
     -1.3735263486386159543e-14,
     2.2082820530301247497e-15,
     -3.3944047611846607383e-16,
     0.0},
    {  // [8, 16], max relative error 9.1e-17
     0.92462581270744814032,
     0.022426046904821617509,
     -0.0033632854246972466529,
     0.00050811207241193898218,
     -0.000077277187286046253259,
     0.000011824509210703231475,
     -1.8193981013257861836e-6,
     2.8137342677733913013e-7,
     -4.3718887142567354835e-8,
     6.8222087358153253457e-9,
     -1.0688256661208552e-9,
     1.6806821429678867679e-10,
     -2.6518258872481906194e-11,
     4.1974007458489564325e-12,
     -6.663421095493081495e-13,
     1.0607424373924901335e-13,
     -1.6929635536870282355e-14,
     2.7102415568166862627e-15,
     -4.4552344095384109015e-16,
     6.9784727943133395388e-17},
    {  // [16, 32], max relative error 1.4e-16
     0.95943546434241239268,
     0.012870093055632837046,
     -0.002047138091502517212,
     0.00032643986998048115045,
     -0.000052177796734008780111,
     8.3586409027615562548e-6,
     -1.3418329765298757476e-6,
     2.1583592432992000242e-7,
     -3.4782826071477127715e-8,
     5.615373870172731813e-9,
     -9.0808208397842418235e-10,
     1.4708451362153951274e-10,
     -2.3859953703679508441e-11,
     3.8761522571891074711e-12,
     -6.305660795720515857e-13,
     1.0271434194219746467e-13,
     -1.6752660181602291294e-14,
     2.7374851966074719439e-15,
     -4.5918922862569621225e-16,
     7.3187533703321782192e-17},
};
// END generated E_1 tables

// sum_{k=1}^{K} (-x)^k / (k k!) by Horner's rule.
__device__ __forceinline__ double e1_series_sum(double x) {
  double s = kE1Series[kE1SeriesTerms - 1];
  #pragma unroll
  for (int k = kE1SeriesTerms - 2; k >= 0; --k) s = fma(s, x, kE1Series[k]);
  return s * x;
}

// x e^x E_1(x) for 1 < x <= 32.
__device__ __forceinline__ double e1_scaled(double x) {
  int e;
  frexp(x, &e);  // x = m 2^e, 1/2 <= m < 1: x in [2^(e-1), 2^e)
  const int seg = min(max(e - 1, 0), 4);
  const double lo = ldexp(1.0, seg), t = (x - lo) / lo * 2.0 - 1.0;  // [lo, 2 lo] -> [-1, 1]
  const double* c = kE1Cheb[seg];
  double b1 = 0.0, b2 = 0.0;
  #pragma unroll
  for (int k = kE1ChebTerms - 1; k >= 1; --k) {
    const double b0 = fma(2.0 * t, b1, c[k] - b2);
    b2 = b1;
    b1 = b0;
  }
  return fma(t, b1, c[0] - b2);
}

__device__ double e1d(double x) {
  if (x <= 1.0) return -kEulerGamma - log(x) - e1_series_sum(x);
  if (x <= 32.0) return e1_scaled(x) * exp(-x) / x;
  const double tiny = 1e-300;
  double b = x + 1.0, c = 1.0 / tiny, d = 1.0 / b, h = d;
  for (int i = 1; i < 200; ++i) {
    const double a = -(double)i * i;
    b += 2.0;
    d = 1.0 / (a * d + b);
    c = b + a / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return h * exp(-x);
}

// psi(a) = 1 + (a - 1) e^{-a} - a^2 E_1(a) (Eq. psi), psi(0) = 0, and its
// first two derivatives: psi' = 2 e^{-a} - 2 a E_1(a), psi'' = -2 E_1(a).
// With R = a e^a E_1(a) for 1 < a <= 32: psi = 1 + e^{-a} ((a - 1) - a R),
// psi' = 2 e^{-a} (1 - R), free of the cancellation in a^2 E_1.
struct Psi3 {
  double v, d1, d2;
};
template <bool D2 = false>
__device__ __forceinline__ Psi3 psid(double a) {
  Psi3 p;
  p.d2 = 0.0;
  if (!(a > 0.0)) {
    p.v = 0.0;
    p.d1 = 2.0;
    p.d2 = -INFINITY;
    return p;
  }
  const double ea = exp(-a);
  if (a > 1.0 && a <= 32.0) {
    const double R = e1_scaled(a);
    p.v = fma(ea, (a - 1.0) - a * R, 1.0);
    p.d1 = 2.0 * ea * (1.0 - R);
    if (D2) p.d2 = -2.0 * ea * R / a;
    return p;
  }
  const double e1 = e1d(a);
  p.v = 1.0 + (a - 1.0) * ea - a * a * e1;
  p.d1 = 2.0 * ea - 2.0 * a * e1;
  if (D2) p.d2 = -2.0 * e1;
  return p;
}

__device__ __forceinline__ size_t fidx(const AL& L, int sp, int i, int j, int x) {
  return (((size_t)sp * 9 + i) * L.N + j) * L.Nx + x;
}
__device__ __forceinline__ bool interior(const AL& L, int x) {
  return L.x_periodic ? (x >= 0 && x < L.Nx) : (x >= 1 && x <= L.Nx - 2);
}
__device__ __forceinline__ int wrapx(const AL& L, int x) {
  if (!L.x_periodic) return x;
  return x < 0 ? x + L.Nx : (x >= L.Nx ? x - L.Nx : x);
}
__device__ __forceinline__ double cwi(const AL& L, int sp, int i) {
  return L.cw[sp][i == 0 ? 0 : (i < 5 ? 1 : 2)];
}

// Per-step column data: r of both walls per column, 1/tau_q of both halves
// per column, kappa of both ends per species.
struct StepCols {
  double* r;      // [2][Nx] bottom, top
  double* omq;    // [2][Nx]
  double* kappa;  // [4]: in_a, in_b, out_a, out_b
  double* dq;     // [4][2][Nx]: d tau_q / d (rho_t, n, alpha, ln mu) per wall node
  double* dr;     // [3][2][Nx]: d r / d (rho_a, rho_b, alpha) per wall node
};
// doubles of one step's column data
__host__ __device__ inline size_t cols_width(int Nx) { return 18 * (size_t)Nx + 4; }

// ----------------------------------------------------------------- pull
// Source value of population i of species sp at (xs, js): the stored state,
// or the virtual ghost column at an end (Eq. rho1, all nine extrapolated and
// scaled by Eq. rho2's kappa).
__device__ double src(const AL& L, const double* f, const double* kap, int sp, int i, int js,
                      int xs) {
  if (!L.x_periodic) {
    if (xs == 0) return kap[sp] * (2.0 * f[fidx(L, sp, i, js, 1)] - f[fidx(L, sp, i, js, 2)]);
    if (xs == L.Nx - 1)
      return kap[2 + sp] *
             (2.0 * f[fidx(L, sp, i, js, L.Nx - 2)] - f[fidx(L, sp, i, js, L.Nx - 3)]);
  }
  return f[fidx(L, sp, i, js, wrapx(L, xs))];
}

// f_i(x) = f'_i(x - c_i) with diffuse bounce-back at rows 0 and N-1: the
// unknowns take (1 - r) of the opposite outgoing population plus r times the
// wall equilibrium with zero normal species flux, 6 w_i (sum of outgoing).
__device__ void pull(const AL& L, const double* f, const double* r2, const double* kap, int x,
                     int j, double g[2][9]) {
  const double rb = r2[x], rt = r2[L.Nx + x];
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    double* q = g[sp];
    q[0] = f[fidx(L, sp, 0, j, x)];
    q[1] = src(L, f, kap, sp, 1, j, x - 1);
    q[3] = src(L, f, kap, sp, 3, j, x + 1);
    if (j == 0) {
      const double o4 = f[fidx(L, sp, 4, j, x)], o7 = f[fidx(L, sp, 7, j, x)],
                   o8 = f[fidx(L, sp, 8, j, x)];
      const double S = o4 + o7 + o8;
      q[2] = (1.0 - rb) * o4 + rb * (2.0 / 3.0) * S;
      q[5] = (1.0 - rb) * o7 + rb * S / 6.0;
      q[6] = (1.0 - rb) * o8 + rb * S / 6.0;
    } else {
      q[2] = f[fidx(L, sp, 2, j - 1, x)];
      q[5] = src(L, f, kap, sp, 5, j - 1, x - 1);
      q[6] = src(L, f, kap, sp, 6, j - 1, x + 1);
    }
    if (j == L.N - 1) {
      const double o2 = f[fidx(L, sp, 2, j, x)], o5 = f[fidx(L, sp, 5, j, x)],
                   o6 = f[fidx(L, sp, 6, j, x)];
      const double S = o2 + o5 + o6;
      q[4] = (1.0 - rt) * o2 + rt * (2.0 / 3.0) * S;
      q[7] = (1.0 - rt) * o5 + rt * S / 6.0;
      q[8] = (1.0 - rt) * o6 + rt * S / 6.0;
    } else {
      q[4] = f[fidx(L, sp, 4, j + 1, x)];
      q[7] = src(L, f, kap, sp, 7, j + 1, x + 1);
      q[8] = src(L, f, kap, sp, 8, j + 1, x - 1);
    }
  }
}

// ------------------------------------------------ node collision (FP64)
// Forward intermediates of one node, kept for the reverse pass.
struct NodeFwd {
  double rho[2], jx[2], jy[2], rho_t, ux, uy, n, mx;
  double inv_rho[2], inv_rt, inv_n, rs_mx, rs_xle[2];  // 1/rho_s, 1/rho, 1/n, m_x^-1/2, xle^-1/2
  double lam, Pm, dPm, tsm, om_s;     // mixture mean free path, Psi, dPsi/dlam, tau_s - 1/2, 1/tau_s
  double lams[2], Ps[2], dPs[2], xle[2], br, d, om_d;
  double m[2][9], meq[2][9];
};

// 1 / |M_k|^2, the diagonal of (M M^T)^-1.
__device__ __forceinline__ double inv_Mnorm(int k) {
  const double w[9] = {1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 6.0, 1.0 / 12.0,
                       1.0 / 6.0, 1.0 / 12.0, 1.0 / 4.0, 1.0 / 4.0};
  return w[k];
}

// m = M v, M the matrix of Eq. m with rows rho, e, eps, j_x, q_x, j_y, q_y,
// p_xx, p_xy, factored over the rest, axis and diagonal classes and their
// sums and differences: 33 FP64 operations instead of one per nonzero entry
// of M (tests/test_adjoint_mrt.py evaluates this code against M).
__device__ __forceinline__ void mrt_fwd(const double v[9], double m[9]) {
  const double a14 = (v[1] + v[2]) + (v[3] + v[4]);
  const double a58 = (v[5] + v[6]) + (v[7] + v[8]);
  m[0] = v[0] + a14 + a58;
  m[1] = fma(-4.0, v[0], fma(2.0, a58, -a14));  // -4 v0 - a14 + 2 a58
  m[2] = fma(4.0, v[0], fma(-2.0, a14, a58));   // 4 v0 - 2 a14 + a58
  const double d13 = v[1] - v[3], d24 = v[2] - v[4];
  const double dx = (v[5] - v[6]) + (v[8] - v[7]);  // diagonal c_x
  const double dy = (v[5] - v[7]) + (v[6] - v[8]);  // diagonal c_y
  m[3] = d13 + dx;
  m[4] = fma(-2.0, d13, dx);
  m[5] = d24 + dy;
  m[6] = fma(-2.0, d24, dy);
  m[7] = (v[1] + v[3]) - (v[2] + v[4]);
  m[8] = (v[5] + v[7]) - (v[6] + v[8]);
}

// o = M^T d, factored the same way (24 FP64 operations).
__device__ __forceinline__ void mrt_tr(const double d[9], double o[9]) {
  o[0] = fma(4.0, d[2] - d[1], d[0]);            // d0 - 4 d1 + 4 d2
  const double B = fma(-2.0, d[2], d[0] - d[1]);  // axis: d0 - d1 - 2 d2
  const double xa = fma(-2.0, d[4], d[3]), ya = fma(-2.0, d[6], d[5]);
  const double Bp = B + d[7], Bm = B - d[7];
  o[1] = Bp + xa;
  o[3] = Bp - xa;
  o[2] = Bm + ya;
  o[4] = Bm - ya;
  const double A = fma(2.0, d[1], d[0] + d[2]);   // diagonal: d0 + 2 d1 + d2
  const double X = d[3] + d[4], Y = d[5] + d[6];
  const double P = A + d[8], Q = A - d[8];
  const double sp = X + Y, sm = X - Y;
  o[5] = P + sp;
  o[7] = P - sp;
  o[6] = Q - sm;
  o[8] = Q + sm;
}

// Psi(y) = (psi(y/lambda) + psi((H-y)/lambda)) / 2 and dPsi/dlambda, from
// 1/lambda.
__device__ __forceinline__ double half_psi(double y, double H, double inv_lam, double* dlam) {
  const Psi3 a = psid(y * inv_lam), b = psid((H - y) * inv_lam);
  *dlam = -0.5 * (a.d1 * y + b.d1 * (H - y)) * inv_lam * inv_lam;
  return 0.5 * (a.v + b.v);
}

// f_out = Collide(g): moments, relaxation rates (1/tau_s of Eq. taos,
// 1/tau_d of Eq. EQFrsp, 1/tau_q from the wall), MRT relaxation
// f' = g - M^{-1} S (m - m^eq).
// psi_in (nullable): the node's Psi and dPsi/dlambda of the mixture and of
// both species as an earlier node_forward stored them through psi_out
// (nullable), six values `plane` doubles apart; read instead of evaluated.
__device__ void node_forward(const AL& L, const double g[2][9], double y, double omq,
                             NodeFwd& F, double fo[2][9], const double* psi_in = nullptr,
                             double* psi_out = nullptr, size_t plane = 0) {
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    mrt_fwd(g[sp], F.m[sp]);  // rho_s, j_x, j_y are rows 0, 3, 5
    F.rho[sp] = F.m[sp][0];
    F.jx[sp] = F.m[sp][3];
    F.jy[sp] = F.m[sp][5];
  }
  F.rho_t = F.rho[0] + F.rho[1];
  F.inv_rt = 1.0 / F.rho_t;
  F.ux = (F.jx[0] + F.jx[1]) * F.inv_rt;
  F.uy = (F.jy[0] + F.jy[1]) * F.inv_rt;
  F.n = L.s[0] * F.rho[0] + L.s[1] * F.rho[1];
  F.inv_n = 1.0 / F.n;
  F.mx = F.rho_t * F.inv_n;
  F.rs_mx = rsqrt(F.mx);
  F.lam = L.c_lam * F.inv_n * F.rs_mx;
  if (psi_in) {
    F.Pm = psi_in[0];
    F.dPm = psi_in[plane];
  } else {
    F.Pm = half_psi(y, L.H, F.n * F.mx * F.rs_mx * L.inv_c_lam, &F.dPm);
  }
  F.tsm = F.lam * F.Pm * L.c_ts * F.rs_mx;
  F.om_s = 1.0 / (0.5 + F.tsm);
  F.br = 0.0;
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    F.inv_rho[sp] = 1.0 / F.rho[sp];
    F.lams[sp] = L.c_xl[sp] / L.s[sp] * F.inv_rho[sp];
    if (psi_in) {
      F.Ps[sp] = psi_in[(2 + 2 * sp) * plane];
      F.dPs[sp] = psi_in[(3 + 2 * sp) * plane];
    } else {
      F.Ps[sp] = half_psi(y, L.H, L.s[sp] * F.rho[sp] * L.inv_c_xl[sp], &F.dPs[sp]);
    }
    F.xle[sp] = L.c_xl[sp] * F.Ps[sp] * F.inv_n;
    F.rs_xle[sp] = rsqrt(F.xle[sp]);
    F.br += F.rs_xle[sp];
  }
  if (psi_out) {
    psi_out[0] = F.Pm;
    psi_out[plane] = F.dPm;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      psi_out[(2 + 2 * sp) * plane] = F.Ps[sp];
      psi_out[(3 + 2 * sp) * plane] = F.dPs[sp];
    }
  }
  F.d = F.mx * F.br * F.br;
  F.om_d = F.d / (0.5 * F.d + L.c_td);
  const double u2 = F.ux * F.ux + F.uy * F.uy;
  const double S[9] = {0.0, L.om_e, L.om_eps, F.om_d, omq, F.om_d, omq, F.om_s, F.om_s};
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const double r = F.rho[sp], s = L.s[sp];
    const double br[9] = {1.0, -4.0 + 2.0 * s + 3.0 * u2, 4.0 - 3.0 * s - 3.0 * u2, F.ux,
                          -F.ux, F.uy, -F.uy, F.ux * F.ux - F.uy * F.uy, F.ux * F.uy};
    double dl[9], c[9];
    #pragma unroll
    for (int k = 0; k < 9; ++k) {
      F.meq[sp][k] = r * br[k];
      dl[k] = S[k] * (F.m[sp][k] - F.meq[sp][k]) * inv_Mnorm(k);
    }
    mrt_tr(dl, c);
    #pragma unroll
    for (int i = 0; i < 9; ++i) fo[sp][i] = g[sp][i] - c[i];
  }
}

// Reverse of node_forward: from fbar (adjoint of f_out) to gbar (adjoint of
// g), omq_bar (adjoint of 1/tau_q) and lnmu_bar (adjoint of ln mu, which
// scales c_lam and c_xl).
__device__ void node_reverse(const AL& L, const double g[2][9], double y, double omq,
                             const double fbar[2][9], double gbar[2][9], double* omq_bar,
                             double* lnmu_bar, const double* psi_in, size_t plane) {
  NodeFwd F;
  double fo[2][9];
  node_forward(L, g, y, omq, F, fo, psi_in, nullptr, plane);
  const double S[9] = {0.0, L.om_e, L.om_eps, F.om_d, omq, F.om_d, omq, F.om_s, F.om_s};
  double Sbar[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  double rhob[2] = {0, 0};
  double uxb = 0, uyb = 0;
  const double u2 = F.ux * F.ux + F.uy * F.uy;
  // adjoint of the moments m = M g; its rows 0, 3, 5 (rho_s, j_x, j_y) also
  // collect the mixture terms below, and gbar = fbar + M^T mbar at the end
  double mbar[2][9];
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const double r = F.rho[sp], s = L.s[sp];
    // f_i = g_i - sum_k M_ki dl_k, dl_k = S_k (m_k - meq_k) / |M_k|^2
    double Mf[9], meqbar[9];
    mrt_fwd(fbar[sp], Mf);
    #pragma unroll
    for (int k = 0; k < 9; ++k) {
      const double dlb = -Mf[k] * inv_Mnorm(k);
      mbar[sp][k] = S[k] * dlb;
      meqbar[k] = -S[k] * dlb;
      Sbar[k] += (F.m[sp][k] - F.meq[sp][k]) * dlb;
    }
    // meq = rho_s (1, -4 + 2s + 3u^2, 4 - 3s - 3u^2, ux, -ux, uy, -uy, ux^2 - uy^2, ux uy)
    const double br[9] = {1.0, -4.0 + 2.0 * s + 3.0 * u2, 4.0 - 3.0 * s - 3.0 * u2, F.ux,
                          -F.ux, F.uy, -F.uy, F.ux * F.ux - F.uy * F.uy, F.ux * F.uy};
    #pragma unroll
    for (int k = 0; k < 9; ++k) rhob[sp] += meqbar[k] * br[k];
    uxb += r * (6.0 * F.ux * (meqbar[1] - meqbar[2]) + meqbar[3] - meqbar[4] +
                2.0 * F.ux * meqbar[7] + F.uy * meqbar[8]);
    uyb += r * (6.0 * F.uy * (meqbar[1] - meqbar[2]) + meqbar[5] - meqbar[6] -
                2.0 * F.uy * meqbar[7] + F.ux * meqbar[8]);
  }
  const double omdb = Sbar[3] + Sbar[5];
  *omq_bar = Sbar[4] + Sbar[6];
  const double omsb = Sbar[7] + Sbar[8];
  double mxb = 0, nb = 0, lnmub = 0;
  // om_d = d / (d/2 + c_td); d = m_x br^2; br = sum_s xle_s^{-1/2}
  const double den = 0.5 * F.d + L.c_td;
  const double db = omdb * L.c_td / (den * den);
  mxb += db * F.br * F.br;
  const double brb = db * 2.0 * F.mx * F.br;
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const double rx = F.rs_xle[sp];
    const double xleb = brb * (-0.5) * rx * rx * rx;
    // xle = c_xl Psi_s / n: proportional to mu through c_xl
    const double Psb = xleb * L.c_xl[sp] * F.inv_n;
    nb -= xleb * F.xle[sp] * F.inv_n;
    lnmub += xleb * F.xle[sp];
    const double lamsb = Psb * F.dPs[sp];
    // lam_s = c_xl / (s rho_s)
    rhob[sp] -= lamsb * F.lams[sp] * F.inv_rho[sp];
    lnmub += lamsb * F.lams[sp];
  }
  // om_s = 1 / (1/2 + tsm); tsm = lam Psi(lam) c_ts m_x^{-1/2}
  const double tsmb = -omsb * F.om_s * F.om_s;
  const double rsm = L.c_ts * F.rs_mx;
  const double inv_mx = F.n * F.inv_rt;
  double lamb = tsmb * (F.Pm + F.lam * F.dPm) * rsm;
  mxb += tsmb * F.tsm * (-0.5) * inv_mx;
  // lam = c_lam n^{-1} m_x^{-1/2}
  nb -= lamb * F.lam * F.inv_n;
  mxb += lamb * F.lam * (-0.5) * inv_mx;
  lnmub += lamb * F.lam;
  // m_x = rho / n; n = sum s rho_s
  double rhotb = mxb * F.inv_n;
  nb -= mxb * F.rho_t * F.inv_n * F.inv_n;
  // u = J / rho
  rhotb -= (uxb * F.ux + uyb * F.uy) * F.inv_rt;
  const double Jxb = uxb * F.inv_rt, Jyb = uyb * F.inv_rt;
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    rhob[sp] += rhotb + nb * L.s[sp];
    mbar[sp][0] += rhob[sp];
    mbar[sp][3] += Jxb;
    mbar[sp][5] += Jyb;
    double c[9];
    mrt_tr(mbar[sp], c);
    #pragma unroll
    for (int i = 0; i < 9; ++i) gbar[sp][i] = fbar[sp][i] + c[i];
  }
  *lnmu_bar = lnmub;
}

// --------------------------------------------------- wall quantities
// Derivatives of tau_q with respect to its inputs (filled by tau_q_rho on
// demand); the reverse of tau_q is these times the adjoint of tau_q.
struct TauqBar {
  double rt;     // rho_t = rho_a + rho_b: d/d g_i for every pulled population
  double n;      // n = sum s rho_s: times s_sigma
  double alpha;  // the accommodation coefficient
  double lnmu;   // ln mu (c_lam is proportional to mu)
};

// tau_q of Eq. taoq from the densities of the pulled wall node (tau'_s(0) in
// its last term, dx = 1) and the accommodation coefficient (Eq. A12); with
// dq != null also its derivatives (reverse mode with a unit adjoint).
// Three FP64 divisions (1/n, 1/tau'(0), 1/alpha); everything else
// multiplies by them.
__device__ double tau_q_rho(const AL& L, double rho0, double rho1, double alpha, TauqBar* dq) {
  const double vs = sqrt(kPiD / 6.0);
  const double rt = rho0 + rho1, n = L.s[0] * rho0 + L.s[1] * rho1;
  const double inv_n = 1.0 / n;
  const double mx = rt * inv_n;
  const double rs = rsqrt(mx);                       // m_x^-1/2
  const double lam = L.c_lam * inv_n * rs;           // mixture mean free path
  const double inv_lam = n * mx * rs * L.inv_c_lam;
  const double gg = L.c_ts * rs;
  const double a = L.H * inv_lam;
  const Psi3 P = psid<true>(a);
  const double tt = 0.5 * lam * P.v * gg;
  const double itt = 1.0 / tt;
  const double i16 = 0.0625 * itt;                   // 1 / (16 tt)
  const double dtt = 0.5 * gg * (2.0 - P.d1);
  const double ial = 1.0 / alpha;
  const double A1 = (2.0 - alpha) * ial * (1.0 - 0.1817 * alpha);
  const double A2 = 1.0 / kPiD + 0.5 * A1 * A1;
  const double Pn = 3.0 + 24.0 * vs * vs * tt * tt * A2;
  const double Qn = 12.0 + 30.0 * tt * vs * A1;
  const double tq = 0.5 + Pn * i16 + dtt * Qn * i16 * itt;
  if (!dq) return tq;
  const double ttb = 48.0 * vs * vs * tt * A2 * i16 - Pn * i16 * itt +
                     dtt * 30.0 * vs * A1 * i16 * itt - 2.0 * dtt * Qn * i16 * itt * itt;
  const double dttb = Qn * i16 * itt;
  const double A2b = 24.0 * vs * vs * tt * tt * i16;
  const double A1b = dtt * 30.0 * vs * i16 + A2b * A1;
  dq->alpha = A1b * ((-2.0 * ial * ial) * (1.0 - 0.1817 * alpha) + (2.0 - alpha) * ial * (-0.1817));
  // tt = lam psi(H/lam) gg / 2, dtt = gg (2 - psi'(H/lam)) / 2
  const double lamb = ttb * 0.5 * gg * (P.v - a * P.d1) + dttb * 0.5 * gg * P.d2 * a * inv_lam;
  const double inv_mx = rs * rs;
  double mxb = (ttb * tt + dttb * dtt) * (-0.5) * inv_mx;
  double nb = -lamb * lam * inv_n;
  mxb += lamb * lam * (-0.5) * inv_mx;
  dq->lnmu = lamb * lam;
  // m_x = rho_t / n
  dq->rt = mxb * inv_n;
  nb -= mxb * rt * inv_n * inv_n;
  dq->n = nb;
  return tq;
}

// r of Eq. R (first form) from the reflected post-collision state of the
// wall node, c_m = c_m0 (2 - alpha)/alpha; dr_drho[2] and dr_dalpha on demand.
__device__ double dbb_r(const AL& L, const double* f, int x, int j, double alpha,
                        double* dr_drho, double* dr_dalpha) {
  double rho[2];
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    rho[sp] = 0;
    #pragma unroll
    for (int i = 0; i < 9; ++i) rho[sp] += f[fidx(L, sp, i, j, x)];
  }
  const double rt = rho[0] + rho[1], n = L.s[0] * rho[0] + L.s[1] * rho[1], mx = rt / n;
  const double cm = L.c_m0 * (2.0 - alpha) / alpha;
  const double q = sqrt(kPiD * mx / 6.0);
  const double den = 1.0 + cm * q;
  if (dr_drho) {
    const double drdmx = 2.0 * cm * (kPiD / 6.0) / (2.0 * q) / (den * den);
    #pragma unroll
    for (int sp = 0; sp < 2; ++sp) dr_drho[sp] = drdmx * (n - rt * L.s[sp]) / (n * n);
    *dr_dalpha = 2.0 * q / (den * den) * L.c_m0 * (-2.0 / (alpha * alpha));
  }
  return 2.0 - 2.0 / den;
}

// ------------------------------------------------------------ kernels
// Sum of v over a block of 256 threads, in a fixed tree order (warp
// shuffles, then the eight warp sums); every thread receives the total.
__device__ double block_sum256(double v, double* sm /* [8] */) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();  // sm may still be read from a previous call
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += sm[k];
  return t;
}

// kappa of both ends (Eq. rho2) from the column sums of columns 1, 2 and
// N_x - 2, N_x - 3 of f; block e (of four) computes kappa[e], e = 2 end +
// species.
__global__ void __launch_bounds__(256) adj_kappa_kernel(AL L, const double* __restrict__ f,
                                                        double* __restrict__ kap) {
  pdl_enter();
  __shared__ double sm[8];
  const int t = threadIdx.x, e = blockIdx.x, sp = e & 1;
  const int x1 = e < 2 ? 1 : L.Nx - 2, x2 = e < 2 ? 2 : L.Nx - 3;
  double a1 = 0.0, a2 = 0.0;
  if (!L.x_periodic) {
    for (int j = t; j < L.N; j += blockDim.x)
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        a1 += f[fidx(L, sp, i, j, x1)];
        a2 += f[fidx(L, sp, i, j, x2)];
      }
  }
  // column sums enter as 2 c(1) - c(2) (resp. N_x - 2, N_x - 3)
  const double D = block_sum256(2.0 * a1 - a2, sm);
  if (t == 0) {
    const double target = e < 2 ? L.rho_in[sp] : L.rho_out[sp];
    kap[e] = L.x_periodic ? 1.0 : L.N * target / D;
  }
}

// r of wall w = blockIdx.y per column, and its derivatives with respect to
// the wall node's species densities and the accommodation coefficient
// (c.dr, for the reverse of the DBB rule).
__global__ void adj_cols_kernel(AL L, const double* __restrict__ f, const double* __restrict__ alpha,
                                StepCols c) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, w = blockIdx.y;
  if (x >= L.Nx) return;
  const size_t k = (size_t)w * L.Nx + x, wn = 2 * (size_t)L.Nx;
  if (!interior(L, x)) {
    c.r[k] = 0.0;
    c.omq[k] = 1.0;
    return;
  }
  double drr[2], dra;
  c.r[k] = dbb_r(L, f, x, w == 0 ? 0 : L.N - 1, alpha[k], drr, &dra);
  c.dr[k] = drr[0];
  c.dr[wn + k] = drr[1];
  c.dr[2 * wn + k] = dra;
}
// 1/tau_q of the half of wall w = blockIdx.y per column, and the
// derivatives of tau_q the reverse sweep multiplies by the adjoint of tau_q
// (c.dq).  One thread per (wall, column): the FP64 pipe takes a warp's 32
// lanes at once, so a thread per wall node is the cheap layout.
__global__ void adj_tauq_kernel(AL L, const double* __restrict__ f, const double* __restrict__ alpha,
                                StepCols c) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x, w = blockIdx.y;
  if (x >= L.Nx || !interior(L, x)) return;
  double g[2][9];
  pull(L, f, c.r, c.kappa, x, w == 0 ? 0 : L.N - 1, g);
  double rho[2];
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    rho[sp] = 0;
    #pragma unroll
    for (int i = 0; i < 9; ++i) rho[sp] += g[sp][i];
  }
  TauqBar d;
  const size_t k = (size_t)w * L.Nx + x, wn = 2 * (size_t)L.Nx;
  c.omq[k] = 1.0 / tau_q_rho(L, rho[0], rho[1], alpha[k], &d);
  c.dq[k] = d.rt;
  c.dq[wn + k] = d.n;
  c.dq[2 * wn + k] = d.alpha;
  c.dq[3 * wn + k] = d.lnmu;
}

// One FP64 step over all nodes: f_out = Collide(Pull(f_in)).  One warp per
// block, block (bx, by) covers 32 columns x `rows` rows (see node_rows).
// psi_out (nullable): [6][N][Nx] Psi values of this step for the reverse
// sweep (see node_forward).  Registers are allocated per SM sub-partition
// (four of 16384): at the 96 this bound leaves (a few values spill to L1)
// each holds five warps, 20 per SM, so one row per block fits the 2560
// warps of a 1280 x 64 channel in one wave on 152 SMs.
__global__ void __launch_bounds__(32, 19) adj_step_kernel(AL L, const double* __restrict__ fin,
                                                      double* __restrict__ fout, StepCols c,
                                                      double* __restrict__ psi_out, int rows) {
  pdl_enter();
  const int x = blockIdx.x * 32 + threadIdx.x;
  if (x >= L.Nx || !interior(L, x)) return;
  const int j0 = blockIdx.y * rows, j1 = min(L.N, j0 + rows);
  const int half = (L.N + 1) / 2;
  const size_t plane = (size_t)L.N * L.Nx;
  for (int j = j0; j < j1; ++j) {
    double g[2][9], fo[2][9];
    pull(L, fin, c.r, c.kappa, x, j, g);
    const double omq = c.omq[(j < half ? 0 : 1) * L.Nx + x];
    NodeFwd F;
    node_forward(L, g, j + 0.5, omq, F, fo, nullptr,
                 psi_out ? psi_out + (size_t)j * L.Nx + x : nullptr, plane);
    #pragma unroll
    for (int sp = 0; sp < 2; ++sp)
      #pragma unroll
      for (int i = 0; i < 9; ++i) fout[fidx(L, sp, i, j, x)] = fo[sp][i];
  }
}

// Initial state (rest equilibrium of the linear pressure and composition
// profiles) and, with dtheta != null, its derivative with respect to theta.
__global__ void adj_init_kernel(AL L, double* __restrict__ f, double* __restrict__ dtheta) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (x >= L.Nx) return;
  const double t = L.x_periodic ? 1.0 : (double)x / (L.Nx - 1);
  const double n = L.x_periodic ? 1.0 : L.theta + (1.0 - L.theta) * t;
  const double dn = L.x_periodic ? 0.0 : 1.0 - t;
  const double Cl = L.C_in + (L.C_out - L.C_in) * t;
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp) {
    const double C = sp == L.light ? Cl : 1.0 - Cl;
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      f[fidx(L, sp, i, j, x)] = cwi(L, sp, i) * n * C * L.mh[sp];
      if (dtheta) dtheta[fidx(L, sp, i, j, x)] = cwi(L, sp, i) * dn * C * L.mh[sp];
    }
  }
}

// Column sums of n_s = s rho_s of a state (for C_l(x)) and of the light
// species' x momentum.
__global__ void adj_colsum_kernel(AL L, const double* __restrict__ f, double* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= L.Nx) return;
  double nl = 0, nh = 0, jl = 0;
  for (int j = 0; j < L.N; ++j)
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      const double a = f[fidx(L, L.light, i, j, x)], b = f[fidx(L, 1 - L.light, i, j, x)];
      nl += L.s[L.light] * a;
      nh += L.s[1 - L.light] * b;
      jl = macc(jl, cxd(i), a);
    }
  out[x] = nl;
  out[L.Nx + x] = nh;
  out[2 * L.Nx + x] = jl;
}

// Adjoint of the objective at the final state: CL = (C_in - C_l(x*))/C_in
// with C_l = S_l / (S_l + S_h) of column x* (objective 0), or the light
// species' x momentum summed over column N_x - 2 (objective 1).
__global__ void adj_seed_kernel(AL L, int objective, int xs, double Sl, double Sh,
                                double* __restrict__ lam) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (x >= L.Nx) return;
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp)
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      double v = 0.0;
      if (objective == 0 && x == xs) {
        const double Sn = Sl + Sh;
        const double dC = sp == L.light ? Sh / (Sn * Sn) : -Sl / (Sn * Sn);
        v = -dC * L.s[sp] / L.C_in;
      } else if (objective == 1 && x == L.Nx - 2 && sp == L.light) {
        v = cxd(i);
      }
      lam[fidx(L, sp, i, j, x)] = v;
    }
}

// Reverse of Collide for every node: gbar = (dCollide/dg)^T lam_t, and
// per node the adjoints of 1/tau_q (of the node's half) and of ln mu,
// stored per row for adj_rev_tauq_kernel to sum in row order:
// part[j][0][x], part[j][1][x].  One warp per block, block (bx, by) covers
// 32 columns x `rows` rows (see node_rows: every block fits on the GPU at
// once, so the SMs share the work to within one block).
// psi: [6][N][Nx] Psi values the forward run or the replay of this step
// stored.  At its 200 registers an SM sub-partition holds two warps, 8 per
// SM, so node_rows gives the 1280 x 64 channel three rows per block (0.72
// waves).  Capped at 168 registers (three warps per sub-partition, two rows
// per block, 40 bytes spilled to L1) it ran 4 % slower.
__global__ void __launch_bounds__(32) adj_rev_node_kernel(
    AL L, const double* __restrict__ fin, const double* __restrict__ lam, StepCols c,
    const double* __restrict__ psi, int rows, double* __restrict__ gbar,
    double* __restrict__ part) {
  pdl_enter();
  const int x = blockIdx.x * 32 + threadIdx.x;
  if (x >= L.Nx || !interior(L, x)) return;
  const int j0 = blockIdx.y * rows, j1 = min(L.N, j0 + rows);
  const int half = (L.N + 1) / 2;
  for (int j = j0; j < j1; ++j) {
    double g[2][9], fb[2][9], gb[2][9];
    pull(L, fin, c.r, c.kappa, x, j, g);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int i = 0; i < 9; ++i) fb[sp][i] = lam[fidx(L, sp, i, j, x)];
    const int h = j < half ? 0 : 1;
    double oqb, lmb;
    node_reverse(L, g, j + 0.5, c.omq[h * L.Nx + x], fb, gb, &oqb, &lmb,
                 psi + (size_t)j * L.Nx + x, (size_t)L.N * L.Nx);
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
      for (int i = 0; i < 9; ++i) gbar[fidx(L, sp, i, j, x)] = gb[sp][i];
    part[(size_t)(2 * j) * L.Nx + x] = oqb;
    part[(size_t)(2 * j + 1) * L.Nx + x] = lmb;
  }
}

// Sum over the warp by a butterfly: every lane gets the same value (each
// stage adds the same two operands in every lane).
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reverse of tau_q per column and wall: one warp per (wall, column), item
// = w N_x + x, kRevTauqWarps per block.  The lanes load the per-row partials
// of adj_rev_node_kernel over the rows of wall w's half (lane-strided, so
// the loads are in flight together) and sum them by a butterfly; then the
// adjoint of tau_q times the derivatives the forward run stored (c.dq) goes
// to the wall node's gbar (lanes 0..17, one population each), the
// accommodation adjoint and ln mu (lnmu_col[w][x]).  The scalar work after
// the sum is a dozen FP64 operations, so its repetition across the lanes
// costs little.
constexpr int kRevTauqWarps = 4;
__global__ void __launch_bounds__(32 * kRevTauqWarps) adj_rev_tauq_kernel(
    AL L, StepCols c, const double* __restrict__ part, double* __restrict__ gbar,
    double* __restrict__ alphabar, double* __restrict__ lnmu_col) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int item = blockIdx.x * kRevTauqWarps + (threadIdx.x >> 5);
  if (item >= 2 * L.Nx) return;  // warp-uniform
  const int w = item >= L.Nx ? 1 : 0, x = item - w * L.Nx;
  if (!interior(L, x)) return;   // warp-uniform
  const int half = (L.N + 1) / 2;
  const int ja = w == 0 ? 0 : half, jb = w == 0 ? half : L.N;
  double omqbar = 0.0, lm = 0.0;
  for (int j = ja + lane; j < jb; j += 32) {
    omqbar += part[(size_t)(2 * j) * L.Nx + x];
    lm += part[(size_t)(2 * j + 1) * L.Nx + x];
  }
  omqbar = warp_sum(omqbar);
  lm = warp_sum(lm);
  const size_t k = (size_t)w * L.Nx + x, wn = 2 * (size_t)L.Nx;
  const double omq = c.omq[k];
  const double taub = -omqbar * omq * omq;  // omq = 1/tau_q
  if (lane < 18) {
    const int sp = lane >= 9 ? 1 : 0;
    const int jw = w == 0 ? 0 : L.N - 1;
    gbar[fidx(L, sp, lane - 9 * sp, jw, x)] += taub * (c.dq[k] + c.dq[wn + k] * L.s[sp]);
  }
  if (lane == 0) {
    alphabar[k] += taub * c.dq[2 * wn + k];
    lnmu_col[k] += lm;
    lnmu_col[k] += taub * c.dq[3 * wn + k];
  }
}

// Transpose of Pull: lam_prev(x, j) gathers the gbar of every node that
// pulled population i of node (x, j) plainly, through the DBB rule of its
// own wall row or through a ghost column, and the DBB rule's r adjoint is
// carried into the wall node's densities and accommodation (with the
// derivatives of r the forward run stored).  Every gather loads from an
// address inside the array whether or not its source exists (the value is
// then dropped), so the loads are independent of one another; the FP64
// work is a few multiply-adds per node, the FP64 pipe being narrow.
// gk: [4] the kappa terms of adj_rev_kappa_kernel, per (end, species).
__global__ void __launch_bounds__(128) adj_rev_pull_kernel(
    AL L, const double* __restrict__ fin, StepCols c, const double* __restrict__ gbar,
    const double* __restrict__ gk, double* __restrict__ lamp, double* __restrict__ alphabar) {
  pdl_enter();
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (x >= L.Nx) return;
  if (!interior(L, x)) {
    #pragma unroll
    for (int sp = 0; sp < 2; ++sp)
      #pragma unroll
      for (int i = 0; i < 9; ++i) lamp[fidx(L, sp, i, j, x)] = 0.0;
    return;
  }
  double lp[2][9];
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp)
    #pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int xd = wrapx(L, x + cxd(i)), jd = j + cyd(i);
      const bool ok = jd >= 0 && jd < L.N && interior(L, xd);
      const double v = gbar[fidx(L, sp, i, ok ? jd : j, ok ? xd : x)];
      lp[sp][i] = ok ? v : 0.0;
    }
  // diffuse bounce-back: the unknowns (2, 5, 6) at row 0 and (4, 7, 8) at
  // row N-1 are pulled from this node's own outgoing populations
  for (int w = 0; w < 2; ++w) {
    const int jw = w == 0 ? 0 : L.N - 1;
    if (j != jw) continue;
    const int unk[3] = {w == 0 ? 2 : 4, w == 0 ? 5 : 7, w == 0 ? 6 : 8};
    const int out[3] = {w == 0 ? 4 : 2, w == 0 ? 7 : 5, w == 0 ? 8 : 6};
    const double r = c.r[w * L.Nx + x];
    double rbar = 0.0;
    #pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const double G0 = gbar[fidx(L, sp, unk[0], j, x)], G1 = gbar[fidx(L, sp, unk[1], j, x)],
                   G2 = gbar[fidx(L, sp, unk[2], j, x)];
      const double o0 = fin[fidx(L, sp, out[0], j, x)], o1 = fin[fidx(L, sp, out[1], j, x)],
                   o2 = fin[fidx(L, sp, out[2], j, x)];
      const double S = o0 + o1 + o2;
      const double T = (2.0 / 3.0) * G0 + (G1 + G2) / 6.0;
      lp[sp][out[0]] += (1.0 - r) * G0 + r * T;
      lp[sp][out[1]] += (1.0 - r) * G1 + r * T;
      lp[sp][out[2]] += (1.0 - r) * G2 + r * T;
      rbar += G0 * (-o0 + (2.0 / 3.0) * S) + G1 * (-o1 + S / 6.0) + G2 * (-o2 + S / 6.0);
    }
    const size_t k = (size_t)w * L.Nx + x, wn = 2 * (size_t)L.Nx;
    #pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const double v = rbar * c.dr[sp * wn + k];
      #pragma unroll
      for (int i = 0; i < 9; ++i) lp[sp][i] += v;
    }
    alphabar[k] += rbar * c.dr[2 * wn + k];
  }
  // the ends: node (x1, jd) pulled population i (c_ix pointing into the
  // channel) from the ghost column kappa (2 f(x1) - f(x2)), and kappa itself
  // depends on the columns x1 = 1, x2 = 2 (N_x - 2, N_x - 3) through gk
  // (adj_rev_kappa_kernel): their transposes land in those columns
  if (!L.x_periodic && (x <= 2 || x >= L.Nx - 3)) {
    #pragma unroll
    for (int end = 0; end < 2; ++end) {
      const int x1 = end == 0 ? 1 : L.Nx - 2, x2 = end == 0 ? 2 : L.Nx - 3;
      if (x != x1 && x != x2) continue;
      const double wgt = x == x1 ? 2.0 : -1.0;
      const int dir = end == 0 ? 1 : -1;
      #pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        const int e = 2 * end + sp;
        const double kap = c.kappa[e];
        #pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int jd = j + cyd(i);
          const bool ok = cxd(i) == dir && jd >= 0 && jd < L.N;
          const double gv = gbar[fidx(L, sp, i, ok ? jd : j, x1)];
          lp[sp][i] += wgt * ((ok ? kap * gv : 0.0) + gk[e]);
        }
      }
    }
  }
  #pragma unroll
  for (int sp = 0; sp < 2; ++sp)
    #pragma unroll
    for (int i = 0; i < 9; ++i) lamp[fidx(L, sp, i, j, x)] = lp[sp][i];
}

// The ends in reverse: the adjoint of kappa_e for (end, species) e = blockIdx.x
// = 2 end + species, reduced over the end columns' rows in a fixed order,
// gives gk[e] = -kappa_bar kappa / D, the weight of d kappa / d f at columns
// x1, x2 (times 2 and -1) that adj_rev_pull_kernel adds, and the inlet's
// theta adjoint (theta_acc[species]).  Threads take (row, population)
// items.
__global__ void __launch_bounds__(256) adj_rev_kappa_kernel(
    AL L, const double* __restrict__ fin, StepCols c, const double* __restrict__ gbar,
    double* __restrict__ gk, double* __restrict__ theta_acc) {
  pdl_enter();
  __shared__ double sm[8];
  const int t = threadIdx.x, e = blockIdx.x;
  if (L.x_periodic) return;
  const int sp = e & 1, inlet = e < 2;
  const int x1 = inlet ? 1 : L.Nx - 2, x2 = inlet ? 2 : L.Nx - 3, dir = inlet ? 1 : -1;
  const double kap = c.kappa[e];
  // node (x1, jd) pulled population i (c_ix = dir) from the ghost column:
  // kappa (2 f(x1, js) - f(x2, js)), js = jd - c_iy
  double acc = 0.0, cs1 = 0.0, cs2 = 0.0;
  for (int k = t; k < 9 * L.N; k += blockDim.x) {
    const int jd = k / 9, i = k - 9 * jd;
    const int js = jd - cyd(i);
    const bool ok = cxd(i) == dir && js >= 0 && js < L.N;
    const int jsc = ok ? js : jd;
    const double gb = gbar[fidx(L, sp, i, jd, x1)];
    const double a1 = fin[fidx(L, sp, i, jsc, x1)], a2 = fin[fidx(L, sp, i, jsc, x2)];
    acc += ok ? gb * (2.0 * a1 - a2) : 0.0;
    cs1 += fin[fidx(L, sp, i, jd, x1)];
    cs2 += fin[fidx(L, sp, i, jd, x2)];
  }
  const double kb = block_sum256(acc, sm);
  const double D = block_sum256(2.0 * cs1 - cs2, sm);
  if (t == 0) {
    // kappa_in = N rho_in / D, rho_in,s = theta C_s m_s
    if (inlet) theta_acc[sp] += kb * kap / L.theta;
    // d kappa / d f(x, j) = -kappa / D * (2 at column x1, -1 at column x2)
    gk[e] = -kb * kap / D;
  }
}

// sum over the state of a * b into one value per block (fixed order); the
// host adds the blocks.
__global__ void adj_dot_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                               double* __restrict__ part) {
  __shared__ double red[256];
  double v = 0;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
       k += (size_t)gridDim.x * blockDim.x)
    v += a[k] * b[k];
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) s += red[k];
    part[blockIdx.x] = s;
  }
}

AL derive_al(const lbm_mix_params* p, int Nx) {
  AL L;
  memset(&L, 0, sizeof L);
  L.N = p->N;
  L.Nx = Nx;
  L.x_periodic = p->x_periodic;
  const double m_min = fmin(p->m_a, p->m_b);
  L.mh[0] = p->m_a / m_min;
  L.mh[1] = p->m_b / m_min;
  L.light = (p->m_a <= p->m_b) ? 0 : 1;
  L.C_in = p->C_l;
  L.C_out = p->C_l_out < 0 ? p->C_l : p->C_l_out;
  L.theta = p->theta;
  double Ci[2], Co[2];
  Ci[L.light] = L.C_in;
  Ci[1 - L.light] = 1.0 - L.C_in;
  Co[L.light] = L.C_out;
  Co[1 - L.light] = 1.0 - L.C_out;
  // mu from lambda_out = Kn_out N at the outlet state (n = 1, p = 1/3)
  const double mx_out = Co[0] * L.mh[0] + Co[1] * L.mh[1];
  const double mu = p->Kn_out * p->N * (1.0 / 3.0) / sqrt(kPiD / (6.0 * mx_out));
  const double mu_s[2] = {p->mu_ratio_a * mu, p->mu_ratio_b * mu};
  for (int sp = 0; sp < 2; ++sp) {
    L.s[sp] = 1.0 / L.mh[sp];
    L.cw[sp][0] = (9.0 - 5.0 * L.s[sp]) / 9.0;
    L.cw[sp][1] = L.s[sp] / 9.0;
    L.cw[sp][2] = L.s[sp] / 36.0;
    L.c_xl[sp] = 3.0 * mu_s[sp] * sqrt(kPiD / (6.0 * L.mh[sp]));
    L.rho_in[sp] = p->theta * Ci[sp] * L.mh[sp];
    L.rho_out[sp] = Co[sp] * L.mh[sp];
  }
  L.c_lam = 3.0 * mu * sqrt(kPiD / 6.0);
  L.inv_c_lam = 1.0 / L.c_lam;
  for (int sp = 0; sp < 2; ++sp) L.inv_c_xl[sp] = 1.0 / L.c_xl[sp];
  L.c_ts = sqrt(6.0 / kPiD);
  L.c_td = 1.5 * sqrt(3.0 * (L.mh[0] + L.mh[1]) * L.mh[0] * L.mh[1]);
  L.om_e = 1.0 / p->tau_e;
  L.om_eps = 1.0 / p->tau_eps;
  L.c_m0 = p->c_m0;
  L.H = p->N;
  return L;
}

}  // namespace

// ------------------------------------------------------------ host side
struct lbm_adj {
  AL L;
  lbm_mix_params p;
  long T = 0;        // steps of the forward run
  int K = 0;         // steps between checkpoints
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t S = 0;      // doubles per state
  double* ckpt = nullptr;   // [ceil(T/K)+1][S] states at steps 0, K, 2K, ...
  int nseg = 0;      // checkpoint intervals, ceil(T/K)
  // Buffer set b (two sets, one when nseg == 1) holds one interval's step
  // inputs, column data and Psi values: the backward sweep replays into
  // them; the forward run fills set (nseg - 1) & 1 with the last interval.
  double* seg[2] = {nullptr, nullptr};      // [K][S] inputs of one segment's steps
  double* segcols[2] = {nullptr, nullptr};  // [K][4 Nx + 4] column data of those steps
  double* segpsi[2] = {nullptr, nullptr};   // [K][6][N][Nx] Psi values of those steps
  cudaStream_t rstream = nullptr;   // the replays of the backward sweep
  cudaEvent_t ev_start = nullptr, ev_rep[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
  double* work[2] = {nullptr, nullptr};
  double* lam[2] = {nullptr, nullptr};
  double* gbar = nullptr;
  double* dtheta0 = nullptr;  // d f^0 / d theta
  double* alpha = nullptr;    // [2][Nx]
  double* alphabar = nullptr;
  double* part_rev = nullptr;  // [N][2][Nx] per-row partials of adj_rev_node_kernel
  int rows_step = 1, rows_rev = 1;  // rows per block of the two node kernels (node_rows)
  double* lnmu_col = nullptr; // [2][Nx] (per wall)
  double* theta_acc = nullptr;  // [2] (per species)
  double* gk = nullptr;         // [4] kappa terms of the step being reversed
  double* colsum = nullptr;   // [3][Nx]
  double* part = nullptr;     // [256]
  double* h_col = nullptr;    // host copy of colsum
  bool have_forward = false;
  bool kept = false;  // set (nseg - 1) & 1 holds the last interval of the forward run
  double CL = 0, flux = 0, Sl = 0, Sh = 0;
  int xstar = -1;
};

namespace {

StepCols cols_of(lbm_adj* a, double* base) {
  StepCols c;
  c.r = base;
  c.omq = base + 2 * a->L.Nx;
  c.kappa = base + 4 * a->L.Nx;
  c.dq = base + 4 * a->L.Nx + 4;
  c.dr = base + 12 * a->L.Nx + 4;
  return c;
}

// Rows per block of a node kernel launched with one-warp blocks of 32
// columns: the fewest rows for which every block is resident at once (the
// occupancy calculator's blocks per SM times the SMs), so that the FP64
// work is spread evenly, with no partial second wave.
cudaError_t node_rows(const void* kernel, int Nx, int N, int* rows) {
  int dev = 0, nsm = 0, occ = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, 32, 0);
  if (e != cudaSuccess) return e;
  const long slots = (long)nsm * (occ > 0 ? occ : 1), ncb = (Nx + 31) / 32;
  int r = 1;
  while (r < N && ncb * ((N + r - 1) / r) > slots) ++r;
  *rows = r;
  return cudaSuccess;
}

// Launches kern with programmatic stream serialisation (see pdl_enter).
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                       Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Forward step from f (input) into fo, column data into cols, on stream st.
int fwd_step(lbm_adj* a, const double* f, double* fo, StepCols c, cudaStream_t st,
             double* psi_out = nullptr) {
  const AL& L = a->L;
  CKA(launch_pdl(adj_kappa_kernel, dim3(4), dim3(256), st, L, f, c.kappa));
  // one thread per (column, wall): small blocks spread the FP64 work of
  // the wall columns over many SMs
  const dim3 wg((L.Nx + 31) / 32, 2);
  CKA(launch_pdl(adj_cols_kernel, wg, dim3(32), st, L, f, (const double*)a->alpha, c));
  CKA(launch_pdl(adj_tauq_kernel, wg, dim3(32), st, L, f, (const double*)a->alpha, c));
  CKA(launch_pdl(adj_step_kernel,
                 dim3((L.Nx + 31) / 32, (L.N + a->rows_step - 1) / a->rows_step), dim3(32), st,
                 L, f, fo, c, psi_out, a->rows_step));
  return LBM_OK;
}

int objective_from_state(lbm_adj* a, const double* f) {
  const AL& L = a->L;
  adj_colsum_kernel<<<(L.Nx + 127) / 128, 128, 0, a->stream>>>(L, f, a->colsum);
  CKA(cudaGetLastError());
  CKA(cudaMemcpyAsync(a->h_col, a->colsum, sizeof(double) * 3 * L.Nx, cudaMemcpyDeviceToHost,
                      a->stream));
  CKA(cudaStreamSynchronize(a->stream));
  // C_l(x) over the updated columns; ties go to the smaller x
  double cmin = INFINITY;
  int xs = -1;
  const int x0 = L.x_periodic ? 0 : 1, x1 = L.x_periodic ? L.Nx - 1 : L.Nx - 2;
  for (int x = x0; x <= x1; ++x) {
    const double C = a->h_col[x] / (a->h_col[x] + a->h_col[L.Nx + x]);
    if (C < cmin) {
      cmin = C;
      xs = x;
    }
  }
  a->xstar = xs;
  a->Sl = a->h_col[xs];
  a->Sh = a->h_col[L.Nx + xs];
  a->CL = (L.C_in - cmin) / L.C_in;
  a->flux = a->h_col[2 * L.Nx + (L.Nx - 2)];
  return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_adj_create(const lbm_mix_params* p, long nsteps, int checkpoint_every, void* stream,
                   lbm_adj** out) {
  if (!out) return lbm_internal_error(LBM_EINVAL, "out is NULL");
  *out = nullptr;
  int Nx = 0;
  int st = lbm_internal_validate(p, &Nx);
  if (st) return st;
  if (nsteps < 1 || checkpoint_every < 1)
    return lbm_internal_error(LBM_EINVAL, "need nsteps >= 1 and checkpoint_every >= 1");
  if (p->x_periodic)
    return lbm_internal_error(LBM_EINVAL, "the adjoint covers channels with pressure ends only");
  if (p->wall != LBM_WALL_DBB)
    return lbm_internal_error(LBM_EINVAL, "the adjoint covers the diffuse bounce-back wall only");
  if (p->r_form != LBM_R_FIRST || p->lambda_pressure != 0)
    return lbm_internal_error(LBM_EINVAL, "the adjoint covers the default readings of Eq. R and "
                                          "of lambda_sigma only");
  lbm_adj* a = new (std::nothrow) lbm_adj;
  if (!a) return lbm_internal_error(LBM_ENOMEM, "host allocation failed");
  a->p = *p;
  a->L = derive_al(p, Nx);
  a->T = nsteps;
  a->K = checkpoint_every < nsteps ? checkpoint_every : (int)nsteps;
  a->S = (size_t)18 * p->N * Nx;
  if (stream) {
    a->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&a->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete a;
      return lbm_internal_error(LBM_ECUDA, "cudaStreamCreate failed");
    }
    a->own_stream = true;
  }
  a->nseg = (int)((nsteps + a->K - 1) / a->K);
  const long nck = a->nseg + 1;
  const size_t cw = cols_width(Nx);
  cudaError_t e = cudaSuccess;
#define ALLOCA(ptr, bytes) \
  if (e == cudaSuccess) e = cudaMalloc((void**)&(ptr), (bytes))
  ALLOCA(a->ckpt, sizeof(double) * a->S * nck);
  for (int b = 0; b < (a->nseg > 1 ? 2 : 1); ++b) {
    ALLOCA(a->seg[b], sizeof(double) * a->S * a->K);
    ALLOCA(a->segcols[b], sizeof(double) * cw * a->K);
    ALLOCA(a->segpsi[b], sizeof(double) * 6 * (size_t)p->N * Nx * a->K);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&a->rstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->ev_start, cudaEventDisableTiming);
  for (int b = 0; b < 2; ++b) {
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->ev_rep[b], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&a->ev_rev[b], cudaEventDisableTiming);
  }
  ALLOCA(a->work[0], sizeof(double) * a->S);
  ALLOCA(a->work[1], sizeof(double) * a->S);
  ALLOCA(a->lam[0], sizeof(double) * a->S);
  ALLOCA(a->lam[1], sizeof(double) * a->S);
  ALLOCA(a->gbar, sizeof(double) * a->S);
  ALLOCA(a->dtheta0, sizeof(double) * a->S);
  ALLOCA(a->alpha, sizeof(double) * 2 * Nx);
  ALLOCA(a->alphabar, sizeof(double) * 2 * Nx);
  ALLOCA(a->part_rev, sizeof(double) * 2 * Nx * (size_t)p->N);
  ALLOCA(a->lnmu_col, sizeof(double) * 2 * Nx);
  ALLOCA(a->theta_acc, sizeof(double) * 2);
  ALLOCA(a->gk, sizeof(double) * 4);
  ALLOCA(a->colsum, sizeof(double) * 3 * Nx);
  ALLOCA(a->part, sizeof(double) * 256);
#undef ALLOCA
  if (e == cudaSuccess) e = cudaMallocHost((void**)&a->h_col, sizeof(double) * (3 * Nx + 256));
  if (e == cudaSuccess) {
    double* al = (double*)malloc(sizeof(double) * 2 * Nx);
    if (!al) {
      e = cudaErrorMemoryAllocation;
    } else {
      for (int k = 0; k < 2 * Nx; ++k) al[k] = p->accommodation;
      e = cudaMemcpyAsync(a->alpha, al, sizeof(double) * 2 * Nx, cudaMemcpyHostToDevice, a->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(a->stream);
      free(al);
    }
  }
  if (e == cudaSuccess) e = node_rows((const void*)adj_step_kernel, Nx, p->N, &a->rows_step);
  if (e == cudaSuccess) e = node_rows((const void*)adj_rev_node_kernel, Nx, p->N, &a->rows_rev);
  if (e != cudaSuccess) {
    const int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    lbm_internal_error(code, "adjoint allocation failed: %s", cudaGetErrorString(e));
    cudaGetLastError();
    lbm_adj_destroy(a);
    return code;
  }
  *out = a;
  return LBM_OK;
}

void lbm_adj_destroy(lbm_adj* a) {
  if (!a) return;
  if (a->stream) cudaStreamSynchronize(a->stream);
  if (a->rstream) cudaStreamSynchronize(a->rstream);
  cudaFree(a->ckpt);
  for (int b = 0; b < 2; ++b) {
    cudaFree(a->seg[b]);
    cudaFree(a->segcols[b]);
    cudaFree(a->segpsi[b]);
    if (a->ev_rep[b]) cudaEventDestroy(a->ev_rep[b]);
    if (a->ev_rev[b]) cudaEventDestroy(a->ev_rev[b]);
  }
  if (a->ev_start) cudaEventDestroy(a->ev_start);
  if (a->rstream) cudaStreamDestroy(a->rstream);
  for (int k = 0; k < 2; ++k) {
    cudaFree(a->work[k]);
    cudaFree(a->lam[k]);
  }
  cudaFree(a->gbar);
  cudaFree(a->dtheta0);
  cudaFree(a->alpha);
  cudaFree(a->alphabar);
  cudaFree(a->part_rev);
  cudaFree(a->lnmu_col);
  cudaFree(a->theta_acc);
  cudaFree(a->gk);
  cudaFree(a->colsum);
  cudaFree(a->part);
  cudaFreeHost(a->h_col);
  if (a->own_stream && a->stream) cudaStreamDestroy(a->stream);
  delete a;
}

int lbm_adj_set_accommodation_field(lbm_adj* a, const double* alpha, long n) {
  if (!a || !alpha) return lbm_internal_error(LBM_EINVAL, "NULL argument");
  if (n != 2L * a->L.Nx) return lbm_internal_error(LBM_EINVAL, "need 2 N_x = %d values", 2 * a->L.Nx);
  for (long k = 0; k < n; ++k)
    if (!(alpha[k] > 0 && alpha[k] <= 1))
      return lbm_internal_error(LBM_EINVAL, "accommodation[%ld] = %g not in (0, 1]", k, alpha[k]);
  CKA(cudaMemcpyAsync(a->alpha, alpha, sizeof(double) * n, cudaMemcpyHostToDevice, a->stream));
  CKA(cudaStreamSynchronize(a->stream));
  a->have_forward = false;
  return LBM_OK;
}

int lbm_adj_forward(lbm_adj* a, double* CL, double* flux) {
  if (!a) return lbm_internal_error(LBM_EINVAL, "handle is NULL");
  const AL& L = a->L;
  const dim3 grd((L.Nx + 127) / 128, L.N);
  adj_init_kernel<<<grd, 128, 0, a->stream>>>(L, a->ckpt, a->dtheta0);
  CKA(cudaGetLastError());
  a->have_forward = false;
  a->kept = false;
  // The last interval's steps keep their inputs, column data and Psi values
  // in buffer set bl, so that the backward sweep need not replay it (with
  // one interval, checkpoint_every >= nsteps, it replays nothing).
  const long tl0 = (long)(a->nseg - 1) * a->K;
  const int bl = (a->nseg - 1) & 1;
  const size_t cw = cols_width(L.Nx), psi_step = 6 * (size_t)L.N * L.Nx;
  const double* f = a->ckpt;
  for (long t = 1; t <= a->T; ++t) {
    double* fo = (t % a->K == 0) ? a->ckpt + a->S * (size_t)(t / a->K) : a->work[t & 1];
    int st;
    if (t > tl0) {
      const long k = t - tl0 - 1;
      if (k == 0)  // f^{tl0} is a checkpoint; the interval's first input
        CKA(cudaMemcpyAsync(a->seg[bl], f, sizeof(double) * a->S, cudaMemcpyDeviceToDevice,
                            a->stream));
      if (t < a->T) fo = a->seg[bl] + a->S * (size_t)(k + 1);
      st = fwd_step(a, a->seg[bl] + a->S * (size_t)k, fo, cols_of(a, a->segcols[bl] + cw * k),
                    a->stream, a->segpsi[bl] + psi_step * (size_t)k);
    } else {
      st = fwd_step(a, f, fo, cols_of(a, a->segcols[0]), a->stream);
    }
    if (st) return st;
    f = fo;
  }
  int st = objective_from_state(a, f);
  if (st) return st;
  if (!isfinite(a->CL)) return lbm_internal_error(LBM_ENONFINITE, "non-finite forward state");
  a->have_forward = true;
  a->kept = true;
  if (CL) *CL = a->CL;
  if (flux) *flux = a->flux;
  return LBM_OK;
}

int lbm_adj_state(lbm_adj* a, double* f, long n) {
  if (!a || !f) return lbm_internal_error(LBM_EINVAL, "NULL argument");
  if (!a->have_forward) return lbm_internal_error(LBM_EINVAL, "run lbm_adj_forward first");
  if (n != (long)a->S) return lbm_internal_error(LBM_EINVAL, "need %zu values", a->S);
  const double* last = (a->T % a->K == 0) ? a->ckpt + a->S * (size_t)(a->T / a->K)
                                           : a->work[a->T & 1];
  CKA(cudaMemcpyAsync(f, last, sizeof(double) * a->S, cudaMemcpyDeviceToHost, a->stream));
  CKA(cudaStreamSynchronize(a->stream));
  return LBM_OK;
}

int lbm_adj_gradient(lbm_adj* a, int objective, double* dtheta, double* dkn, double* dalpha,
                     long n_alpha) {
  if (!a) return lbm_internal_error(LBM_EINVAL, "handle is NULL");
  if (objective != LBM_ADJ_CL && objective != LBM_ADJ_FLUX)
    return lbm_internal_error(LBM_EINVAL, "unknown objective %d", objective);
  if (!a->have_forward) return lbm_internal_error(LBM_EINVAL, "run lbm_adj_forward first");
  const AL& L = a->L;
  if (dalpha && n_alpha != 2L * L.Nx)
    return lbm_internal_error(LBM_EINVAL, "dalpha needs 2 N_x = %d values", 2 * L.Nx);
  const dim3 grd((L.Nx + 127) / 128, L.N);
  const size_t cw = cols_width(L.Nx);
  CKA(cudaMemsetAsync(a->alphabar, 0, sizeof(double) * 2 * L.Nx, a->stream));
  CKA(cudaMemsetAsync(a->lnmu_col, 0, sizeof(double) * 2 * L.Nx, a->stream));
  CKA(cudaMemsetAsync(a->theta_acc, 0, sizeof(double) * 2, a->stream));
  adj_seed_kernel<<<grd, 128, 0, a->stream>>>(L, objective, a->xstar, a->Sl, a->Sh, a->lam[0]);
  CKA(cudaGetLastError());
  int cur = 0;  // lam[cur] is the adjoint of the state after the step being reversed
  const long nseg = a->nseg;
  // the replay's last output of a segment is not needed (only its column
  // data are); it goes to the work buffer that does not hold f^T, so that
  // lbm_adj_state still returns the forward run's final state afterwards
  double* spare = a->work[1 - (a->T & 1)];
  // Replay of segment sg (inputs f^{t0} .. f^{t1-1}, their column data and
  // Psi values) into buffer set sg & 1, on the replay stream.
  const size_t psi_step = 6 * (size_t)L.N * L.Nx;
  auto replay = [&](long sg) -> int {
    const int b = (int)(sg & 1);
    const long t0 = sg * a->K, t1 = (t0 + a->K < a->T) ? t0 + a->K : a->T;
    CKA(cudaMemcpyAsync(a->seg[b], a->ckpt + a->S * (size_t)sg, sizeof(double) * a->S,
                        cudaMemcpyDeviceToDevice, a->rstream));
    for (long t = t0 + 1; t <= t1; ++t) {
      const long k = t - t0 - 1;
      double* fin = a->seg[b] + a->S * (size_t)k;
      double* fo = (t < t1) ? a->seg[b] + a->S * (size_t)(k + 1) : spare;
      int st = fwd_step(a, fin, fo, cols_of(a, a->segcols[b] + cw * k), a->rstream,
                        a->segpsi[b] + psi_step * (size_t)k);
      if (st) return st;
    }
    CKA(cudaEventRecord(a->ev_rep[b], a->rstream));
    return LBM_OK;
  };
  // The replay of segment sg - 1 runs on the replay stream while segment
  // sg is reversed on the handle's stream (double-buffered); a replay waits
  // for the reverse that last used its buffer pair, a reverse for its
  // replay.  Each kernel computes what it did in sequence, so the gradient
  // is the same bit for bit.
  CKA(cudaEventRecord(a->ev_start, a->stream));
  CKA(cudaStreamWaitEvent(a->rstream, a->ev_start, 0));
  // the forward run left the last interval in its buffer set
  const bool last_kept = a->kept;
  int st0 = last_kept ? LBM_OK : replay(nseg - 1);
  if (st0) return st0;
  // a replay into the last interval's set (segment nseg - 3, ...) ends it
  if (nseg >= 3) a->kept = false;
  for (long sg = nseg - 1; sg >= 0; --sg) {
    const int b = (int)(sg & 1);
    if (sg >= 1) {
      if (sg + 1 <= nseg - 1) CKA(cudaStreamWaitEvent(a->rstream, a->ev_rev[(sg + 1) & 1], 0));
      if ((st0 = replay(sg - 1))) return st0;
    }
    if (!(last_kept && sg == nseg - 1)) CKA(cudaStreamWaitEvent(a->stream, a->ev_rep[b], 0));
    const long t0 = sg * a->K;
    const long t1 = (t0 + a->K < a->T) ? t0 + a->K : a->T;
    for (long t = t1; t > t0; --t) {
      const long k = t - t0 - 1;
      const double* fin = a->seg[b] + a->S * (size_t)k;
      StepCols c = cols_of(a, a->segcols[b] + cw * k);
      CKA(launch_pdl(adj_rev_node_kernel,
                     dim3((L.Nx + 31) / 32, (L.N + a->rows_rev - 1) / a->rows_rev), dim3(32),
                     a->stream, L, fin, (const double*)a->lam[cur], c,
                     (const double*)(a->segpsi[b] + psi_step * (size_t)k), a->rows_rev, a->gbar,
                     a->part_rev));
      CKA(launch_pdl(adj_rev_tauq_kernel, dim3((2 * L.Nx + kRevTauqWarps - 1) / kRevTauqWarps),
                     dim3(32 * kRevTauqWarps), a->stream, L, c, (const double*)a->part_rev,
                     a->gbar, a->alphabar, a->lnmu_col));
      // one block per (end, species); the pull adds its kappa terms
      CKA(launch_pdl(adj_rev_kappa_kernel, dim3(4), dim3(256), a->stream, L, fin, c,
                     (const double*)a->gbar, a->gk, a->theta_acc));
      CKA(launch_pdl(adj_rev_pull_kernel, grd, dim3(128), a->stream, L, fin, c,
                     (const double*)a->gbar, (const double*)a->gk, a->lam[1 - cur], a->alphabar));
      cur = 1 - cur;
    }
    CKA(cudaEventRecord(a->ev_rev[b], a->stream));
  }
  // theta through the initial state: lam^0 . d f^0 / d theta
  adj_dot_kernel<<<256, 256, 0, a->stream>>>(a->lam[cur], a->dtheta0, a->S, a->part);
  CKA(cudaGetLastError());
  double* h = a->h_col;  // staging: [2][Nx] ln mu, [2] theta, [256] parts
  CKA(cudaMemcpyAsync(h, a->lnmu_col, sizeof(double) * 2 * L.Nx, cudaMemcpyDeviceToHost,
                      a->stream));
  CKA(cudaMemcpyAsync(h + 2 * L.Nx, a->theta_acc, sizeof(double) * 2, cudaMemcpyDeviceToHost,
                      a->stream));
  CKA(cudaMemcpyAsync(h + 2 * L.Nx + 2, a->part, sizeof(double) * 256, cudaMemcpyDeviceToHost,
                      a->stream));
  if (dalpha)
    CKA(cudaMemcpyAsync(dalpha, a->alphabar, sizeof(double) * 2 * L.Nx, cudaMemcpyDeviceToHost,
                        a->stream));
  CKA(cudaStreamSynchronize(a->stream));
  double lnmu = 0, th = h[2 * L.Nx] + h[2 * L.Nx + 1];
  for (int x = 0; x < 2 * L.Nx; ++x) lnmu += h[x];
  for (int k = 0; k < 256; ++k) th += h[2 * L.Nx + 2 + k];
  if (dtheta) *dtheta = th;
  if (dkn) *dkn = lnmu / a->p.Kn_out;  // mu is proportional to Kn_out
  return LBM_OK;
}

}  // extern "C"
