// Device code of the DMN material-point update (sm_103a).
//
// One thread owns one Gauss point.  The tree is traversed depth first with an
// explicit per-thread stack: on the way down the laminate jumps are corrected
// (top-down redistribution of the previous Newton step) and the leaf strains
// are formed; at the leaves the phase laws give stress and tangent; on the way
// up every laminate is condensed (bottom-up homogenisation of the linearised
// problem) and its share of the Newton residual is accumulated.  All threads
// of a warp walk the same tree in lock step, so tree parameters are read at
// warp-uniform addresses.
//
// Laminates are indexed in heap order inside this file (root h = 1, children
// 2h and 2h + 1, array index h - 1); the paper's ordering (level K first, root
// last) is used only at the ABI (state jumps, p, q).
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#ifndef DMN_HOST_EMULATION
#include <cuda_runtime.h>
#endif

namespace dmn {

constexpr int KMAX = 8;
constexpr int NMAX = (1 << KMAX) - 1;
constexpr double RS2 = 0.70710678118654752440;   // 1/sqrt(2)
constexpr double SQ23 = 0.81649658092772603273;  // sqrt(2/3)
// The mixed forms' all-FP32 first stage: Newton passes in FP32 until
// ||A^T W sigma|| <= STAGE_TOL (2^K - 1) ||sigma_bar|| (its FP32 residual) or STAGE_MAX_ITER
// corrections; the FP64-residual iteration continues from its jumps.
constexpr float STAGE_TOL = 1e-8f;
constexpr int STAGE_MAX_ITER = 12;

// Isotropic phase: elastic (kind 0), J2 with linear isotropic hardening
// (kind 1) or with exponential-linear hardening (kind 2, Sec. 4.1):
//   sigma_Y(a) = s0 + H a + ds (1 - exp(-rate a)),  ds = sigma_inf - s0,
//   rate = (k0 - H) / ds,  slope sigma_Y'(a) = H + (k0 - H) exp(-rate a).
// Constants derived once on the host.
struct PhaseDev {
  int kind;
  double K, G;       // bulk and shear modulus
  double s0, H;      // yield stress and (linear part of the) hardening modulus
  double lam;        // K - 2G/3: sigma = lam tr(eps) 1 + 2G eps when elastic
  float lamf, Gf;    // FP32 copies of lam and G (elastic leaf tangents of the FP32 form)
  double inv_den;    // 1 / (2G + 2H/3): plastic multiplier per unit overstress (kind 1)
  double thb0;       // 1 / (1 + H / (3G)) (kind 1)
  double ds, dk, rate;  // kind 2: sigma_inf - s0, k0 - H, (k0 - H) / (sigma_inf - s0)
  // FP32 copies of the constants above, for the all-FP32 passes of the mixed forms' first stage
  struct {
    float K, G, s0, H, lam, inv_den, thb0, ds, dk, rate;
  } f;
};

// Per-laminate constants, heap order.
struct TreeDev {
  int K, M, N, L;
  int nz;            // inelastic leaves
  int z_both;        // 1 if both phases are inelastic (slot = leaf), else slot = leaf / 2
  const double* p;   // [N][M]
  const double* q;   // [N][M]
  const double* c1;  // [N] volume fraction of the left child
  const double* c2;  // [N] volume fraction of the right child
  const double* sc;  // [N] W c1 c2: scale of the laminate's residual (W = subtree weight)
  const float* c1f;  // [N] FP32 copies of c1, c2, c1 c2
  const float* c2f;
  const float* c12f;
  const float* scf;  // [N] FP32 copy of sc
  const double* ic12;  // [N] 1 / (c1 c2): the stored Newton step is c1 c2 (g, H), see condense
  const float* ic12f;  // [N] FP32 copy
  const double* wl;  // [L] normalised leaf weights
  double wsum;       // sum of the leaf weights as given
  PhaseDev ph[2];
  // Compressed traversal (tree compression, Sec. 3.1: leaves of weight zero
  // removed, a laminate with one weightless subtree replaced by the other
  // subtree).  The laminates are then numbered in the paper's order among the
  // remaining ones (p, q, c1, ... follow that numbering, N counts them) and the
  // tree is walked by tables instead of heap arithmetic.
  int Lc;            // leaves with weight > 0, in leaf order
  const int4* lf;    // per such leaf: x = depth where its descent starts, y = laminates descended to reach it,
                     // z = laminates completed right after it,
                     // w = leaf << 12 | (state slot + 1) << 2 | phase << 1 | pair,
                     // pair = 1 when this leaf and the next are the two children of one laminate
  const int* pre;    // [N] laminates in descent (pre-) order
  const int* post;   // [N] laminates in completion (post-) order
  const int* pidx;   // [N] the paper's index of each laminate (in the uncompressed tree)
  const int* kid;    // [2 N] children of each laminate: >= 0 a laminate, -1 - phase a leaf
  const int* hcid;   // [2^K - 1] the laminate standing at each heap position, -1 for none (compressed trees)
  const int* kslot;  // [2 N] the state slot of each child that is a leaf (-1: elastic, or a laminate child)
};

// fields of TreeDev::lf .w
__device__ __forceinline__ int lf_slot(int w) { return ((w >> 2) & 1023) - 1; }
__device__ __forceinline__ int lf_phase(int w) { return (w >> 1) & 1; }
__device__ __forceinline__ int lf_leaf(int w) { return w >> 12; }

template <typename T>
struct NodeC {
  T c1, c2, c12;
};
// 1 / (c1 c2) of a laminate in precision T
template <typename T>
__device__ __forceinline__ T ic12_of(const TreeDev& t, int node);
template <>
__device__ __forceinline__ double ic12_of<double>(const TreeDev& t, int node) { return __ldg(t.ic12 + node); }
template <>
__device__ __forceinline__ float ic12_of<float>(const TreeDev& t, int node) { return __ldg(t.ic12f + node); }
template <typename T>
__device__ __forceinline__ NodeC<T> node_c(const TreeDev& t, int node);
template <>
__device__ __forceinline__ NodeC<double> node_c<double>(const TreeDev& t, int node) {
  const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
  return {c1, c2, c1 * c2};
}
template <>
__device__ __forceinline__ NodeC<float> node_c<float>(const TreeDev& t, int node) {
  return {__ldg(t.c1f + node), __ldg(t.c2f + node), __ldg(t.c12f + node)};
}

// ---------------------------------------------------------------------------
// Conversions between FP64 and the working precision T.  For T = float they
// work on the IEEE 754 binary64 / binary32 bit patterns with integer
// instructions: GB300 executes a hardware FP64 <-> FP32 conversion on its FP64
// pipe, at 1/64 of the rate of the FP32 and integer pipes, and the FP32 form
// converts some 3000 values per tree pass.
//   narrow_rn: round to nearest, ties to even; results below the smallest
//              normal FP32 number (2^-126) become a signed zero; overflow
//              gives infinity, NaN stays NaN.
//   widen:     exact; FP32 subnormals become a signed zero.
// (host and device: the host build lets a CPU test compare them with the host's IEEE conversions)
__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned bits_of(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned u;
  memcpy(&u, &x, sizeof u);
  return u;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  memcpy(&x, &u, sizeof x);
  return x;
#endif
}
__host__ __device__ __forceinline__ float narrow_rn(double x) {
  const unsigned long long b = bits_of(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const unsigned e = (hi >> 20) & 0x7ffu;                      // biased exponent (bias 1023)
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);   // the 23 leading fraction bits
  const unsigned rest = lo & 0x1fffffffu;                      // the 29 fraction bits rounded away
  unsigned r = ((e - 896u) << 23) + mant;                      // bias 127; a rounding carry may reach the exponent
  r += (rest > 0x10000000u || (rest == 0x10000000u && (mant & 1u))) ? 1u : 0u;
  if (e <= 896u) r = 0u;
  if (e >= 1151u) r = (e == 2047u && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
  return float_of(sign | r);
}
__host__ __device__ __forceinline__ double widen(float x) {
  const unsigned u = bits_of(x);
  const unsigned e = (u >> 23) & 0xffu;
  unsigned hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
  unsigned lo = u << 29;
  if (e == 0u) {
    hi = u & 0x80000000u;
    lo = 0u;
  } else if (e == 255u) {
    hi = (u & 0x80000000u) | 0x7ff00000u | ((u & 0x7fffffu) >> 3);
  }
  return double_of((unsigned long long)hi << 32 | lo);
}
__device__ __forceinline__ double widen(double x) { return x; }
template <typename T>
__device__ __forceinline__ T narrow(double x);
template <>
__device__ __forceinline__ double narrow<double>(double x) { return x; }
template <>
__device__ __forceinline__ float narrow<float>(double x) { return narrow_rn(x); }
// a constant held in both precisions
template <typename T>
__device__ __forceinline__ T pick(double d, float f);
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }

// x converted to T: exact or by narrow_rn / widen (integer instructions), never by a hardware conversion
template <typename T, typename S>
struct Cvt;
template <>
struct Cvt<double, double> { __host__ __device__ static double f(double x) { return x; } };
template <>
struct Cvt<float, double> { __host__ __device__ static float f(double x) { return narrow_rn(x); } };
template <>
struct Cvt<float, float> { __host__ __device__ static float f(float x) { return x; } };
template <>
struct Cvt<double, float> { __host__ __device__ static double f(float x) { return widen(x); } };
template <typename T, typename S>
__device__ __forceinline__ T cvt(S x) { return Cvt<T, S>::f(x); }

// a parameter type that takes no part in template argument deduction (a NULL argument then fits)
template <typename X>
struct NoDeduce { using type = X; };

// the math functions in precision S (float: the FP32 versions, so that nothing runs on the FP64 pipe)
__device__ __forceinline__ double rsqrt_s(double x) { return rsqrt(x); }
__device__ __forceinline__ float rsqrt_s(float x) { return rsqrtf(x); }
__device__ __forceinline__ double sqrt_s(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_s(float x) { return sqrtf(x); }
__device__ __forceinline__ double exp_s(double x) { return exp(x); }
__device__ __forceinline__ float exp_s(float x) { return expf(x); }
__device__ __forceinline__ double fabs_s(double x) { return fabs(x); }
__device__ __forceinline__ float fabs_s(float x) { return fabsf(x); }
__device__ __forceinline__ double fmax_s(double x, double y) { return fmax(x, y); }
__device__ __forceinline__ float fmax_s(float x, float y) { return fmaxf(x, y); }
// smallest squared norm taken as non-zero, and a value above any relative yield gap
template <typename S>
__device__ __forceinline__ S tiny_s();
template <>
__device__ __forceinline__ double tiny_s<double>() { return 1e-300; }
template <>
__device__ __forceinline__ float tiny_s<float>() { return 1e-36f; }
template <typename S>
__device__ __forceinline__ S huge_s();
template <>
__device__ __forceinline__ double huge_s<double>() { return 1e300; }
template <>
__device__ __forceinline__ float huge_s<float>() { return 1e30f; }

// packed symmetric 6x6: upper triangle row by row
__host__ __device__ constexpr int sidx(int i, int j) {
  return i <= j ? i * 6 - (i * (i - 1)) / 2 + (j - i) : j * 6 - (j * (j - 1)) / 2 + (i - j);
}

// Result of a subtree.  Its linearised response to a strain perturbation d_eps,
// with its inner jumps re-equilibrated, is sb + ds + C d_eps: sb is the plain
// weighted-average stress at the current iterate (FP64; it also feeds the
// residual), ds the change that the inner Newton corrections add (precision
// T), C the condensed tangent (T).  Keeping sb apart in FP64 lets the FP32
// form see the residual, a small difference of large stresses, exactly.
// The all-FP32 passes (S = float) keep sb in FP32 as well.
template <typename T, typename S = double>
struct Sub {
  S sb[6];
  T ds[6];
  T C[21];
};

// Tangent of an isotropic leaf: D = lam 1(x)1 + 2 mu I - c m(x)m.
template <typename T>
struct LeafTan {
  T lam, mu, c;
  T m[6];
};

// ---------------------------------------------------------------------------
// Phase law (Sec. 3.2 condensed GSM leaf; Sec. 4.1 J2 radial return with
// isotropic hardening sigma_Y).  z = (alpha_bar, ep11, ep22, ep23M, ep13M, ep12M).
//   xi = dev eps - ep, s_tr = 2G xi, f = |s_tr| - sqrt(2/3) sigma_Y(alpha_bar);
//   f > 0: dg from |s_tr| - 2G dg = sqrt(2/3) sigma_Y(alpha_bar + sqrt(2/3) dg)
//          (linear law: dg = f / (2G + 2H/3)), n = xi / |xi|, s = (1 - k2) s_tr
//          with k2 = 2G dg / |s_tr| = dg / |xi|, ep += dg n, alpha_bar += sqrt(2/3) dg,
//          D = K 1(x)1 + 2G th Idev - 2G thb n(x)n, th = 1 - k2,
//          thb = 1/(1 + sigma_Y'/(3G)) - (1 - th).
// Written without branches: an elastic step is the plastic formula with dg = 0.
// S: the precision of strains, state and stress (double; float in the mixed forms' all-FP32
// first stage, whose constants are the phase's FP32 copies).
template <typename T, typename S = double>
__device__ __forceinline__ void leaf_iso(const PhaseDev& ph, const S e[6], const S z[6], S sig[6], LeafTan<T>* D,
                                         typename NoDeduce<S>::type* znew, typename NoDeduce<S>::type* gap) {
  const S K = pick<S>(ph.K, ph.f.K), G = pick<S>(ph.G, ph.f.G), lam = pick<S>(ph.lam, ph.f.lam);
  const S tr = e[0] + e[1] + e[2];
  const S twoG = (S)2 * G;
  if (ph.kind == 0) {
    const S lt = lam * tr;
#pragma unroll
    for (int I = 0; I < 6; ++I) sig[I] = twoG * e[I];
    sig[0] += lt; sig[1] += lt; sig[2] += lt;
    if (D) {
      D->lam = pick<T>(ph.lam, ph.lamf); D->mu = pick<T>(ph.G, ph.Gf); D->c = (T)0;
#pragma unroll
      for (int I = 0; I < 6; ++I) D->m[I] = (T)0;
    }
    if (gap) *gap = huge_s<S>();
    return;
  }
  const S s0 = pick<S>(ph.s0, ph.f.s0), H = pick<S>(ph.H, ph.f.H);
  const S sq23 = (S)SQ23;
  const S m3 = tr * (S)(1.0 / 3.0);
  const S ep2 = -(z[1] + z[2]);
  const S xi[6] = {e[0] - m3 - z[1], e[1] - m3 - z[2], e[2] - m3 - ep2, e[3] - z[3], e[4] - z[4], e[5] - z[5]};
  S n2 = (S)0;
#pragma unroll
  for (int I = 0; I < 6; ++I) n2 += xi[I] * xi[I];
  const S inx = rsqrt_s(fmax_s(n2, tiny_s<S>()));   // 1 / |xi|
  const S ns = twoG * (n2 * inx);                    // |s_tr|
  const bool explin = ph.kind == 2;
  const S rate = pick<S>(ph.rate, ph.f.rate), dsat = pick<S>(ph.ds, ph.f.ds), dk = pick<S>(ph.dk, ph.f.dk);
  const S e_n = explin ? exp_s(-rate * z[0]) : (S)1;
  const S sy = s0 + H * z[0] + (explin ? dsat * ((S)1 - e_n) : (S)0);
  const S f = ns - sq23 * sy;
  const bool plastic = f > (S)0;
  if (gap) *gap = fabs_s(f) / sy;
  S dg = plastic ? f * pick<S>(ph.inv_den, ph.f.inv_den) : (S)0;
  S thb0 = pick<S>(ph.thb0, ph.f.thb0);
  if (explin && plastic) {
    // scalar Newton on r(dg) = |s_tr| - 2G dg - sqrt(2/3) sigma_Y(a_n + sqrt(2/3) dg).  r is convex and
    // decreasing, so from dg = 0 the iterates rise monotonically to the root; the first iterate,
    // f / (2G + 2/3 sigma_Y'(a_n)), needs no new exponential.  Convergence is quadratic, so once a
    // step is below 1e-10 dg the next would be below the rounding of dg: stop there.  In FP32 the
    // residual's rounding bounds a step from below by about 1e-7 |xi|: stop at 1e-6 dg + 2e-7 |xi|.
    S slope = H + dk * e_n, ex = e_n, step = (S)0;
    dg = f / (twoG + (S)(2.0 / 3.0) * slope);
    const S floor_abs = sizeof(S) == 8 ? (S)0 : (S)2e-7f * (n2 * inx);
    const S rel = sizeof(S) == 8 ? (S)1e-10 : (S)1e-6f;
    for (int it = 0; it < 40; ++it) {
      const S a = z[0] + sq23 * dg;
      ex = exp_s(-rate * a);
      slope = H + dk * ex;
      const S r = ns - twoG * dg - sq23 * (s0 + H * a + dsat * ((S)1 - ex));
      step = r / (twoG + (S)(2.0 / 3.0) * slope);
      dg += step;
      if (sizeof(S) == 8 ? fabs_s(step) <= rel * dg : fabs_s(step) <= rel * dg + floor_abs) break;
    }
    // hardening slope at the new a: the last one was taken one step earlier; its first-order
    // correction -rate dk e sqrt(2/3) step leaves an error of order (rate step)^2
    slope -= rate * dk * ex * sq23 * step;
    thb0 = (S)1 / ((S)1 + slope / ((S)3 * G));
  }
  const S k2 = dg * inx;          // 2G dg / |s_tr| = 1 - th
  const S Kt = K * tr;
  const S g2 = twoG - twoG * k2;  // 2G th
#pragma unroll
  for (int I = 0; I < 6; ++I) sig[I] = g2 * xi[I];
  sig[0] += Kt; sig[1] += Kt; sig[2] += Kt;
  if (D) {
    const S mu = G * ((S)1 - k2);
    D->mu = cvt<T>(mu);
    D->lam = cvt<T>(K - (S)(2.0 / 3.0) * mu);
    D->c = cvt<T>(plastic ? twoG * (thb0 - k2) : (S)0);
    if (sizeof(T) == sizeof(S)) {
#pragma unroll
      for (int I = 0; I < 6; ++I) D->m[I] = cvt<T>(xi[I] * inx);
    } else {   // the FP32 tangent's flow direction, normalised in FP32
      const T it = cvt<T>(inx);
#pragma unroll
      for (int I = 0; I < 6; ++I) D->m[I] = cvt<T>(xi[I]) * it;
    }
  }
  if (znew) {
    znew[0] = z[0] + sq23 * dg;         // ep += dg n = k2 xi
    znew[1] = z[1] + k2 * xi[0]; znew[2] = z[2] + k2 * xi[1];
    znew[3] = z[3] + k2 * xi[3]; znew[4] = z[4] + k2 * xi[4]; znew[5] = z[5] + k2 * xi[5];
  }
}

// ---------------------------------------------------------------------------
// N(n) a = sym(a (x) n) in Mandel form, and N^T v = v n (as a tensor).
template <typename T>
__device__ __forceinline__ void N_apply(const T n[3], const T nr[3], const T a[3], T out[6]) {
  out[0] = n[0] * a[0];
  out[1] = n[1] * a[1];
  out[2] = n[2] * a[2];
  out[3] = nr[2] * a[1] + nr[1] * a[2];
  out[4] = nr[2] * a[0] + nr[0] * a[2];
  out[5] = nr[1] * a[0] + nr[0] * a[1];
}
template <typename T>
__device__ __forceinline__ void Nt_apply(const T n[3], const T nr[3], const T v[6], T out[3]) {
  out[0] = n[0] * v[0] + nr[2] * v[4] + nr[1] * v[5];
  out[1] = n[1] * v[1] + nr[2] * v[3] + nr[0] * v[5];
  out[2] = n[2] * v[2] + nr[1] * v[3] + nr[0] * v[4];
}
// S N for packed symmetric S: 6x3
template <typename T>
__device__ __forceinline__ void SN_apply(const T S[21], const T n[3], const T nr[3], T out[6][3]) {
#pragma unroll
  for (int I = 0; I < 6; ++I) {
    out[I][0] = S[sidx(I, 0)] * n[0] + S[sidx(I, 4)] * nr[2] + S[sidx(I, 5)] * nr[1];
    out[I][1] = S[sidx(I, 1)] * n[1] + S[sidx(I, 3)] * nr[2] + S[sidx(I, 5)] * nr[0];
    out[I][2] = S[sidx(I, 2)] * n[2] + S[sidx(I, 3)] * nr[1] + S[sidx(I, 4)] * nr[0];
  }
}
// structural non-zeros of N: (I, I) for I < 3 and two entries in each shear row
__host__ __device__ constexpr bool N_nonzero(int I, int j) {
  return I < 3 ? I == j : !((I == 3 && j == 0) || (I == 4 && j == 1) || (I == 5 && j == 2));
}
// entry (I, j) of N: column j of sym(e_j (x) n)
template <typename T>
__device__ __forceinline__ T N_entry(const T n[3], const T nr[3], int I, int j) {
  if (I < 3) return I == j ? n[j] : (T)0;
  const int a = I == 3 ? 1 : 0, b = I == 5 ? 1 : 2;  // index pair of shear component I
  if (j == a) return nr[b];
  if (j == b) return nr[a];
  return (T)0;
}

// Symmetric 3x3 inverse by cofactors (the matrix is positive definite), times s.
template <typename T>
__device__ __forceinline__ void inv3_sym(T k00, T k01, T k02, T k11, T k12, T k22, T Ki[3][3], T s = (T)1) {
  const T i00 = k11 * k22 - k12 * k12;
  const T i01 = k02 * k12 - k01 * k22;
  const T i02 = k01 * k12 - k02 * k11;
  const T i11 = k00 * k22 - k02 * k02;
  const T i12 = k01 * k02 - k00 * k12;
  const T i22 = k00 * k11 - k01 * k01;
  const T idet = s / (k00 * i00 + k01 * i01 + k02 * i02);
  Ki[0][0] = i00 * idet; Ki[0][1] = i01 * idet; Ki[0][2] = i02 * idet;
  Ki[1][0] = Ki[0][1];   Ki[1][1] = i11 * idet; Ki[1][2] = i12 * idet;
  Ki[2][0] = Ki[0][2];   Ki[2][1] = Ki[1][2];   Ki[2][2] = i22 * idet;
}

// The laminate's FP64 residual share (A^T W sigma)_j = W c1 c2 N^T (sb_R - sb_L),
// added to r2, the plain average sb = c1 sb_L + c2 sb_R, and t = N^T (sb_R - sb_L).
// (In the all-FP32 first stage, S = float, it is the FP32 residual of that stage.)
template <typename S>
__device__ __forceinline__ void residual_share(const S nd[3], S c1, S c2, S sc, const S sL[6], const S sR[6], S sb[6],
                                               S t[3], S& r2) {
  S d[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) d[I] = sR[I] - sL[I];
  const S ndr[3] = {nd[0] * (S)RS2, nd[1] * (S)RS2, nd[2] * (S)RS2};
  Nt_apply<S>(nd, ndr, d, t);
  r2 += sc * sc * (t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
#pragma unroll
  for (int I = 0; I < 6; ++I) sb[I] = sL[I] + c2 * d[I];   // c1 sL + c2 sR with c1 = 1 - c2
}

// The plain average alone, sb = c1 sb_L + c2 sb_R (as residual_share forms it): the final sweep,
// which needs the stress and the tangent but neither the residual nor a Newton step.
template <typename S>
__device__ __forceinline__ void stress_average(S c2, const S sL[6], const S sR[6], S sb[6]) {
#pragma unroll
  for (int I = 0; I < 6; ++I) sb[I] = sL[I] + c2 * (sR[I] - sL[I]);
}

// ---------------------------------------------------------------------------
// Condensation of one laminate with children L (fraction c1) and R (c2) and
// normal n.  Jumps perturb the children as d_eps_L = d_eps - c2 N da,
// d_eps_R = d_eps + c1 N da (Sec. 3.2, gradient operator); equilibrium
// N^T (sigma_R - sigma_L) = 0 of the linearised children gives
//   Kn da = -N^T (s_R - s_L) - B^T d_eps,  Kn = N^T (c2 C_L + c1 C_R) N,
//   B = (C_R - C_L) N,
// i.e. da = g + H d_eps with g = -Kn^-1 N^T (s_R - s_L), H = -Kn^-1 B^T, and
// the laminate's affine response
//   s = c1 s_L + c2 s_R + c1 c2 B g,  C = c1 C_L + c2 C_R + c1 c2 B H,
// with s = sb + ds split as in Sub: N^T (s_R - s_L) = t + N^T (ds_R - ds_L),
// t = N^T (sb_R - sb_L) taken from the FP64 residual.
// For constant child tangents this is the laminate homogenisation of Sec. 3.1;
// eliminating laminates leaves-to-root is Gaussian elimination of the Newton
// system A^T W D A da = -A^T W sigma of Sec. 3.2 (no fill in that order).
template <typename T, bool STORE, typename S = double>
__device__ __forceinline__ void condense(const S nd[3], const T n[3], S c1d, S c2d, S sc, NodeC<T> cc,
                                         const Sub<T, S>& L, const Sub<T, S>& R, Sub<T, S>& out, T* gp,
                                         size_t gstride, S& r2) {
  // without STORE (the final sweep) only sb and C: no residual, no Newton step g, no ds
  T u[3] = {(T)0, (T)0, (T)0};
  if (STORE) {
    S t[3];
    residual_share<S>(nd, c1d, c2d, sc, L.sb, R.sb, out.sb, t, r2);
    u[0] = cvt<T>(t[0]); u[1] = cvt<T>(t[1]); u[2] = cvt<T>(t[2]);
  } else {
    stress_average<S>(c2d, L.sb, R.sb, out.sb);
  }
  const T c1 = cc.c1, c2 = cc.c2, c12 = cc.c12;
  const T nr[3] = {n[0] * (T)RS2, n[1] * (T)RS2, n[2] * (T)RS2};
  // c2 C_L + c1 C_R = C_R - c2 dC and c1 X_L + c2 X_R = X_L + c2 dX with c1 = 1 - c2: one
  // fused multiply-add per entry
  T Ch[21], dC[21];
#pragma unroll
  for (int k = 0; k < 21; ++k) { dC[k] = R.C[k] - L.C[k]; Ch[k] = R.C[k] - c2 * dC[k]; }
  T ChN[6][3], B[6][3];
  SN_apply<T>(Ch, n, nr, ChN);
  SN_apply<T>(dC, n, nr, B);
  // Kn = N^T (C-hat N), symmetric: its six distinct entries, row i of N^T against column m
  const T k00 = n[0] * ChN[0][0] + nr[2] * ChN[4][0] + nr[1] * ChN[5][0];
  const T k10 = n[1] * ChN[1][0] + nr[2] * ChN[3][0] + nr[0] * ChN[5][0];
  const T k20 = n[2] * ChN[2][0] + nr[1] * ChN[3][0] + nr[0] * ChN[4][0];
  const T k11 = n[1] * ChN[1][1] + nr[2] * ChN[3][1] + nr[0] * ChN[5][1];
  const T k21 = n[2] * ChN[2][1] + nr[1] * ChN[3][1] + nr[0] * ChN[4][1];
  const T k22 = n[2] * ChN[2][2] + nr[1] * ChN[3][2] + nr[0] * ChN[4][2];
  // the inverse times c1 c2: H and g come out as c1 c2 H, c1 c2 g, so that the condensed outputs
  // are multiply-add chains; the descent multiplies the step by 1 / (c1 c2)
  T Ki[3][3];
  inv3_sym<T>(k00, k10, k20, k11, k21, k22, Ki, c12);
  T H[3][6];   // c1 c2 H
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int I = 0; I < 6; ++I) H[m][I] = -(Ki[m][0] * B[I][0] + Ki[m][1] * B[I][1] + Ki[m][2] * B[I][2]);
  T dds[6], v[3], g[3];   // g: c1 c2 g
  if (STORE) {
#pragma unroll
    for (int I = 0; I < 6; ++I) dds[I] = R.ds[I] - L.ds[I];
    Nt_apply<T>(n, nr, dds, v);
#pragma unroll
    for (int m = 0; m < 3; ++m) u[m] += v[m];
#pragma unroll
    for (int m = 0; m < 3; ++m) g[m] = -(Ki[m][0] * u[0] + Ki[m][1] * u[1] + Ki[m][2] * u[2]);
#pragma unroll
    for (int I = 0; I < 6; ++I)
      out.ds[I] = L.ds[I] + c2 * dds[I] + B[I][0] * g[0] + B[I][1] * g[1] + B[I][2] * g[2];
  } else {
#pragma unroll
    for (int I = 0; I < 6; ++I) out.ds[I] = (T)0;
  }
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = I; J < 6; ++J) {
      const int s = sidx(I, J);
      T v = L.C[s] + c2 * dC[s];
      v += B[I][0] * H[0][J];
      v += B[I][1] * H[1][J];
      v += B[I][2] * H[2][J];
      out.C[s] = v;
    }
  if (STORE) {
#pragma unroll
    for (int m = 0; m < 3; ++m) gp[m * gstride] = g[m];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int I = 0; I < 6; ++I) gp[(3 + 6 * m + I) * gstride] = H[m][I];
  }
}

// Condensation of a bottom laminate, whose children are leaves with isotropic
// tangents D_X = lam_X 1(x)1 + 2 mu_X I - c_X m_X (x) m_X (X = L, R).  With
// N^T 1 = n and N^T N = (I + n (x) n) / 2 the laminate algebra above reduces to
//   Kn = a I + b n (x) n - c2 c_L u_L (x) u_L - c1 c_R u_R (x) u_R,
//        a = c2 mu_L + c1 mu_R, b = c2 (lam_L + mu_L) + c1 (lam_R + mu_R), u_X = N^T m_X,
//   B  = (lam_R - lam_L) 1 (x) n + 2 (mu_R - mu_L) N - c_R m_R (x) u_R + c_L m_L (x) u_L,
//   C  = (c1 lam_L + c2 lam_R) 1(x)1 + 2 (c1 mu_L + c2 mu_R) I
//        - c1 c_L m_L (x) m_L - c2 c_R m_R (x) m_R + c1 c2 B H,
// and, the leaves having no inner corrections, ds = c1 c2 B g with g = -Kn^-1 t.
// A leaf of an elastic phase has c_X = 0 in every pass: elL / elR (the phases of the
// tree's left and right leaves, the same for every lane) drop its rank-one terms in the
// FP64 condensation, which leaves every non-zero result unchanged.
template <typename T, bool STORE, typename S = double>
__device__ __forceinline__ void condense_bottom(const S nd[3], const T n[3], S c1d, S c2d, S sc, NodeC<T> cc,
                                                const S sL[6], const LeafTan<T>& DL, const S sR[6],
                                                const LeafTan<T>& DR, Sub<T, S>& out, T* gp, size_t gstride, S& r2,
                                                bool elL, bool elR) {
  // the FP32 condensation runs beside the FP64 work at no cost of its own: it keeps the general
  // form, whose register use the shortcut would raise
  if (sizeof(T) == 4) { elL = false; elR = false; }
  T u[3] = {(T)0, (T)0, (T)0};
  if (STORE) {
    S t[3];
    residual_share<S>(nd, c1d, c2d, sc, sL, sR, out.sb, t, r2);
    u[0] = cvt<T>(t[0]); u[1] = cvt<T>(t[1]); u[2] = cvt<T>(t[2]);
  } else {
    stress_average<S>(c2d, sL, sR, out.sb);
  }
  const T c1 = cc.c1, c2 = cc.c2, c12 = cc.c12;
  const T nr[3] = {n[0] * (T)RS2, n[1] * (T)RS2, n[2] * (T)RS2};
  T uL[3], uR[3];
  const T a = c2 * DL.mu + c1 * DR.mu;
  const T b = c2 * (DL.lam + DL.mu) + c1 * (DR.lam + DR.mu);
  T k[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) k[i][j] = b * n[i] * n[j] + (i == j ? a : (T)0);
  T cmL[6], cmR[6];
  if (!elL) {
    Nt_apply<T>(n, nr, DL.m, uL);
    const T wL = c2 * DL.c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) k[i][j] -= wL * uL[i] * uL[j];
#pragma unroll
    for (int I = 0; I < 6; ++I) cmL[I] = DL.c * DL.m[I];
  }
  if (!elR) {
    Nt_apply<T>(n, nr, DR.m, uR);
    const T wR = c1 * DR.c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) k[i][j] -= wR * uR[i] * uR[j];
#pragma unroll
    for (int I = 0; I < 6; ++I) cmR[I] = DR.c * DR.m[I];
  }
  T Ki[3][3];   // times c1 c2, as in condense
  inv3_sym<T>(k[0][0], k[0][1], k[0][2], k[1][1], k[1][2], k[2][2], Ki, c12);
  // (lam_R - lam_L) 1 (x) n + 2 (mu_R - mu_L) N: entry (I, j) is dlam n_j (I < 3, j != I),
  // (dlam + dmu2) n_j (I = j) or dmu2 N_Ij (shear rows)
  const T dlam = DR.lam - DL.lam, dmu2 = (T)2 * (DR.mu - DL.mu), dld = dlam + dmu2;
  T B[6][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      B[I][j] = I < 3 ? (I == j ? dld : dlam) * n[j] : (N_nonzero(I, j) ? dmu2 * N_entry<T>(n, nr, I, j) : (T)0);
  if (!elL) {
#pragma unroll
    for (int I = 0; I < 6; ++I)
#pragma unroll
      for (int j = 0; j < 3; ++j) B[I][j] += cmL[I] * uL[j];
  }
  if (!elR) {
#pragma unroll
    for (int I = 0; I < 6; ++I)
#pragma unroll
      for (int j = 0; j < 3; ++j) B[I][j] -= cmR[I] * uR[j];
  }
  T H[3][6];   // c1 c2 H
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int I = 0; I < 6; ++I) H[m][I] = -(Ki[m][0] * B[I][0] + Ki[m][1] * B[I][1] + Ki[m][2] * B[I][2]);
  T g[3] = {(T)0, (T)0, (T)0};   // c1 c2 g
  if (STORE) {
#pragma unroll
    for (int m = 0; m < 3; ++m) g[m] = -(Ki[m][0] * u[0] + Ki[m][1] * u[1] + Ki[m][2] * u[2]);
#pragma unroll
    for (int I = 0; I < 6; ++I) out.ds[I] = B[I][0] * g[0] + B[I][1] * g[1] + B[I][2] * g[2];
  } else {
#pragma unroll
    for (int I = 0; I < 6; ++I) out.ds[I] = (T)0;
  }
  const T lamC = c1 * DL.lam + c2 * DR.lam, mu2C = (T)2 * (c1 * DL.mu + c2 * DR.mu);
  T Cb[21];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = I; J < 6; ++J) {
      T v = B[I][0] * H[0][J] + B[I][1] * H[1][J] + B[I][2] * H[2][J];
      if (I < 3 && J < 3) v += lamC;
      if (I == J) v += mu2C;
      Cb[sidx(I, J)] = v;
    }
  if (!elL) {
    T hL[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) hL[I] = c1 * cmL[I];
#pragma unroll
    for (int I = 0; I < 6; ++I)
#pragma unroll
      for (int J = I; J < 6; ++J) Cb[sidx(I, J)] -= hL[I] * DL.m[J];
  }
  if (!elR) {
    T hR[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) hR[I] = c2 * cmR[I];
#pragma unroll
    for (int I = 0; I < 6; ++I)
#pragma unroll
      for (int J = I; J < 6; ++J) Cb[sidx(I, J)] -= hR[I] * DR.m[J];
  }
#pragma unroll
  for (int k2 = 0; k2 < 21; ++k2) out.C[k2] = Cb[k2];
  if (STORE) {
#pragma unroll
    for (int m = 0; m < 3; ++m) gp[m * gstride] = g[m];
#pragma unroll
    for (int m = 0; m < 3; ++m)
#pragma unroll
      for (int I = 0; I < 6; ++I) gp[(3 + 6 * m + I) * gstride] = H[m][I];
  }
}

// ---------------------------------------------------------------------------
// Per-thread views of strided arrays.
struct PointArrays {
  const double* nrm; size_t ns;  // normals: element (3*node + c) at nrm[(3*node+c)*ns]
  const float* nrmf;             // FP32 copy of the normals (same indexing; FP32 form only)
  double* a; size_t as;          // jumps: a[(3*j+c)*as], j = node (heap) or the paper's index
  double* a_out;                 // where corrected jumps are written (same indexing; == a: in place)
  bool paper;                    // jumps stored in the paper's ordering (level K first, root last)
  const double* z; size_t zs;    // leaf state z^n of the inelastic slots: z[(6*slot+c)*zs]
  float* af;                     // the all-FP32 passes: jumps in FP32 (indexing of a)
  float* af_out;
};

// Per-laminate and per-leaf inputs of a pass in its state precision S: the FP32 passes read the
// FP32 copies (normals, volume fractions) or narrow the FP64 values with integer instructions
// (leaf states).
template <typename S>
struct PassIn;
template <>
struct PassIn<double> {
  __device__ static double* a(const PointArrays& P) { return P.a; }
  __device__ static double* a_out(const PointArrays& P) { return P.a_out; }
  __device__ static double c1(const TreeDev& t, int j) { return __ldg(t.c1 + j); }
  __device__ static double c2(const TreeDev& t, int j) { return __ldg(t.c2 + j); }
  __device__ static double sc(const TreeDev& t, int j) { return __ldg(t.sc + j); }
};
template <>
struct PassIn<float> {
  __device__ static float* a(const PointArrays& P) { return P.af; }
  __device__ static float* a_out(const PointArrays& P) { return P.af_out; }
  __device__ static float c1(const TreeDev& t, int j) { return __ldg(t.c1f + j); }
  __device__ static float c2(const TreeDev& t, int j) { return __ldg(t.c2f + j); }
  __device__ static float sc(const TreeDev& t, int j) { return __ldg(t.scf + j); }
};

// array index of the jumps of heap node `node` at level lvl
__device__ __forceinline__ int jump_index(const PointArrays& P, int K, int lvl, int node) {
  return P.paper ? (1 << K) - 3 * (1 << (lvl - 1)) + node + 1 : node;
}

template <typename T>
struct GH {
  T* p; size_t s;  // c1 c2 g and c1 c2 H of laminate node read by a pass: p[(21*node + c)*s], c = 0..2 g, 3..20 H
  T* q;            // where the pass stores the new g and H (== p: in place)
};

template <typename T>
__device__ __forceinline__ void load_n(const PointArrays& P, int node, double nd[3], T n[3]);
template <>
__device__ __forceinline__ void load_n<double>(const PointArrays& P, int node, double nd[3], double n[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) { nd[c] = P.nrm[(3 * node + c) * P.ns]; n[c] = nd[c]; }
}
template <>
__device__ __forceinline__ void load_n<float>(const PointArrays& P, int node, double nd[3], float n[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) { nd[c] = P.nrm[(3 * node + c) * P.ns]; n[c] = P.nrmf[(3 * node + c) * P.ns]; }
}

// normals in the state precision S and in the working precision T
template <typename T, typename S>
__device__ __forceinline__ void load_ns(const PointArrays& P, int node, S nd[3], T n[3]) {
  if (sizeof(S) == 8) {
    load_n<T>(P, node, reinterpret_cast<double*>(nd), n);
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) { n[c] = (T)P.nrmf[(3 * node + c) * P.ns]; nd[c] = (S)n[c]; }
  }
}

template <typename S>
__device__ __forceinline__ void load_z(const TreeDev& t, const PointArrays& P, int leaf, int phase, S z[6]) {
  if (t.ph[phase].kind != 0) {
    const int slot = t.z_both ? leaf : (leaf >> 1);
    const double* b = P.z + (size_t)(6 * slot) * P.zs;
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = cvt<S>(b[c * P.zs]);
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = (S)0;
  }
}

// One pass over the tree for one point.
//   STORE:  Newton pass.  When `apply` is set, first apply the previous Newton
//           step scaled by `step` on the way down, da = step g + H d_eps with the
//           g, H stored by the previous pass, a_out = a + da (top-down
//           redistribution; the scaled step is the same linear map applied to
//           step g); then store this pass's g, H for the next step (both times c1 c2: the
//           descent applies 1 / (c1 c2) to the step).
//   !STORE: evaluation at the given jumps only (final sweep).
// Returns the root's subtree result (sb = effective stress, C = tangent of the
// linearised DMN) and the squared norm of A^T W sigma at the (updated) jumps.
// S: the precision of strains, jumps, leaf stresses and residual (double; float in the mixed
// forms' all-FP32 first stage, which reads and writes the FP32 jumps af).
template <typename T, bool STORE, typename S = double>
__device__ void tree_pass(const TreeDev& t, const S Eloc[6], const PointArrays& P, GH<T> gh, bool apply, T step,
                          Sub<T, S>& root, S& r2, typename NoDeduce<S>::type* gap_min) {
  const int K = t.K;
  S epsR[KMAX + 1][6];
  T depsR[KMAX + 1][6];
  Sub<T, S> pend[KMAX + 1];
  r2 = (S)0;
  S* const a_in = PassIn<S>::a(P);
  S* const a_wr = PassIn<S>::a_out(P);
  const int nbottom = 1 << (K - 1);
  for (int m = 0; m < nbottom; ++m) {
    const int top = (m == 0) ? 1 : K - __ffs(m) + 1;
    S e[6];
    T de[6];
    if (m == 0) {
#pragma unroll
      for (int I = 0; I < 6; ++I) { e[I] = Eloc[I]; de[I] = (T)0; }
    } else {
#pragma unroll
      for (int I = 0; I < 6; ++I) { e[I] = epsR[top][I]; de[I] = depsR[top][I]; }
    }
    S eL[6], eR[6];
    for (int lvl = top; lvl <= K; ++lvl) {
      const int node = (1 << (lvl - 1)) + (m >> (K - lvl)) - 1;
      S nd[3];
      T nt[3];
      load_ns<T, S>(P, node, nd, nt);
      const S c1 = PassIn<S>::c1(t, node), c2 = PassIn<S>::c2(t, node);
      const size_t aoff = (size_t)(3 * jump_index(P, K, lvl, node)) * P.as;
      const S* ap = a_in + aoff;
      S a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      T da[3] = {(T)0, (T)0, (T)0};
      if (STORE) {   // only the Newton kernel corrects jumps; `apply` is false on a point's first pass
        const T* gp = gh.p + (size_t)(21 * node) * gh.s;
        const T ic = ic12_of<T>(t, node);   // the stored step is c1 c2 (g, H)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T v = step * gp[c * gh.s];
#pragma unroll
          for (int I = 0; I < 6; ++I) v += gp[(3 + 6 * c + I) * gh.s] * de[I];
          da[c] = apply ? v * ic : (T)0;
        }
        S* aw = a_wr + aoff;
#pragma unroll
        for (int c = 0; c < 3; ++c) { a[c] += cvt<S>(da[c]); aw[c * P.as] = a[c]; }
      }
      const S ndr[3] = {nd[0] * (S)RS2, nd[1] * (S)RS2, nd[2] * (S)RS2};
      S Na[6];
      N_apply<S>(nd, ndr, a, Na);
#pragma unroll
      for (int I = 0; I < 6; ++I) { eL[I] = e[I] - c2 * Na[I]; eR[I] = e[I] + c1 * Na[I]; }
      if (lvl < K) {
        T dR[6];
        if (STORE) {
          const NodeC<T> cc = node_c<T>(t, node);
          const T ntr[3] = {nt[0] * (T)RS2, nt[1] * (T)RS2, nt[2] * (T)RS2};
          T Nda[6];
          N_apply<T>(nt, ntr, da, Nda);
#pragma unroll
          for (int I = 0; I < 6; ++I) { dR[I] = de[I] + cc.c1 * Nda[I]; de[I] = de[I] - cc.c2 * Nda[I]; }
        } else {
#pragma unroll
          for (int I = 0; I < 6; ++I) dR[I] = (T)0;
        }
#pragma unroll
        for (int I = 0; I < 6; ++I) { epsR[lvl + 1][I] = eR[I]; depsR[lvl + 1][I] = dR[I]; e[I] = eL[I]; }
      }
    }
    // leaves 2m (phase 1) and 2m + 1 (phase 2), condensed by their bottom laminate
    Sub<T, S> res;
    {
      const int node = nbottom + m - 1;
      S z[6], g, sL[6], sR[6];
      LeafTan<T> DL, DR;
      load_z<S>(t, P, 2 * m, 0, z);
      leaf_iso<T, S>(t.ph[0], eL, z, sL, &DL, nullptr, gap_min ? &g : nullptr);
      if (gap_min) *gap_min = fmin(*gap_min, g);
      load_z<S>(t, P, 2 * m + 1, 1, z);
      leaf_iso<T, S>(t.ph[1], eR, z, sR, &DR, nullptr, gap_min ? &g : nullptr);
      if (gap_min) *gap_min = fmin(*gap_min, g);
      S nd[3];
      T nt[3];
      load_ns<T, S>(P, node, nd, nt);
      T* gp = STORE ? gh.q + (size_t)(21 * node) * gh.s : nullptr;
      condense_bottom<T, STORE, S>(nd, nt, PassIn<S>::c1(t, node), PassIn<S>::c2(t, node), PassIn<S>::sc(t, node),
                                   node_c<T>(t, node), sL, DL, sR, DR, res, gp, gh.s, r2, t.ph[0].kind == 0,
                                   t.ph[1].kind == 0);
    }
    // condense upwards while the finished laminate is a right child
    int lvl = K, idx = m;
    for (;;) {
      if (lvl == 1) { root = res; break; }
      if (!(idx & 1)) { pend[lvl] = res; break; }
      idx >>= 1;
      --lvl;
      const int node = (1 << (lvl - 1)) + idx - 1;
      S nd[3];
      T nt[3];
      load_ns<T, S>(P, node, nd, nt);
      T* gp = STORE ? gh.q + (size_t)(21 * node) * gh.s : nullptr;
      const Sub<T, S> B = res;
      condense<T, STORE, S>(nd, nt, PassIn<S>::c1(t, node), PassIn<S>::c2(t, node), PassIn<S>::sc(t, node),
                            node_c<T>(t, node), pend[lvl + 1], B, res, gp, gh.s, r2);
    }
  }
}

// Tangent and stress of one leaf as a subtree result (no inner jumps).
template <typename T, typename S = double>
__device__ __forceinline__ void leaf_sub(const LeafTan<T>& D, const S sig[6], Sub<T, S>& s) {
#pragma unroll
  for (int I = 0; I < 6; ++I) { s.sb[I] = sig[I]; s.ds[I] = (T)0; }
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = I; J < 6; ++J) {
      T v = -D.c * D.m[I] * D.m[J];
      if (I < 3 && J < 3) v += D.lam;
      if (I == J) v += (T)2 * D.mu;
      s.C[sidx(I, J)] = v;
    }
}

template <typename S>
__device__ __forceinline__ void load_z_slot(const PointArrays& P, int slot, S z[6]) {
  if (slot >= 0) {
    const double* b = P.z + (size_t)(6 * slot) * P.zs;
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = cvt<S>(b[c * P.zs]);
  } else {
#pragma unroll
    for (int c = 0; c < 6; ++c) z[c] = (S)0;
  }
}

// The pass of tree_pass over a compressed tree, driven by the tables of
// TreeDev (laminates by their compressed number; jumps at that number in both
// the scratch and the state).  Same arithmetic per laminate and leaf; a leaf
// whose sibling is a laminate enters the condensation as a subtree with the
// leaf's tangent, two sibling leaves use the structured bottom condensation.
template <typename T, bool STORE, typename S = double>
__device__ void tree_pass_c(const TreeDev& t, const S Eloc[6], const PointArrays& P, GH<T> gh, bool apply, T step,
                            Sub<T, S>& root, S& r2, typename NoDeduce<S>::type* gap_min) {
  S epsR[KMAX + 1][6];
  T depsR[KMAX + 1][6];
  Sub<T, S> pend[KMAX + 1];
  r2 = (S)0;
  S* const a_in = PassIn<S>::a(P);
  S* const a_wr = PassIn<S>::a_out(P);
  int ipre = 0, ipost = 0;
  for (int l = 0; l < t.Lc;) {
    const int4 f = __ldg(t.lf + l);
    const bool pair = f.w & 1;
    int d = f.x;
    S e[6];
    T de[6];
    if (l == 0) {
#pragma unroll
      for (int I = 0; I < 6; ++I) { e[I] = Eloc[I]; de[I] = (T)0; }
    } else {
#pragma unroll
      for (int I = 0; I < 6; ++I) { e[I] = epsR[d][I]; de[I] = depsR[d][I]; }
    }
    for (int s = 0; s < f.y; ++s, ++d) {
      const int node = __ldg(t.pre + ipre++);
      S nd[3];
      T nt[3];
      load_ns<T, S>(P, node, nd, nt);
      const S c1 = PassIn<S>::c1(t, node), c2 = PassIn<S>::c2(t, node);
      const S* ap = a_in + (size_t)(3 * node) * P.as;
      S a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      T da[3] = {(T)0, (T)0, (T)0};
      if (STORE) {
        const T* gp = gh.p + (size_t)(21 * node) * gh.s;
        const T ic = ic12_of<T>(t, node);   // the stored step is c1 c2 (g, H)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T v = step * gp[c * gh.s];
#pragma unroll
          for (int I = 0; I < 6; ++I) v += gp[(3 + 6 * c + I) * gh.s] * de[I];
          da[c] = apply ? v * ic : (T)0;
        }
        S* aw = a_wr + (size_t)(3 * node) * P.as;
#pragma unroll
        for (int c = 0; c < 3; ++c) { a[c] += cvt<S>(da[c]); aw[c * P.as] = a[c]; }
      }
      const S ndr[3] = {nd[0] * (S)RS2, nd[1] * (S)RS2, nd[2] * (S)RS2};
      S Na[6];
      N_apply<S>(nd, ndr, a, Na);
      T dR[6];
      if (STORE && !(pair && s == f.y - 1)) {   // children that are laminates need strain corrections
        const NodeC<T> cc = node_c<T>(t, node);
        const T ntr[3] = {nt[0] * (T)RS2, nt[1] * (T)RS2, nt[2] * (T)RS2};
        T Nda[6];
        N_apply<T>(nt, ntr, da, Nda);
#pragma unroll
        for (int I = 0; I < 6; ++I) { dR[I] = de[I] + cc.c1 * Nda[I]; de[I] = de[I] - cc.c2 * Nda[I]; }
      } else {
#pragma unroll
        for (int I = 0; I < 6; ++I) dR[I] = (T)0;
      }
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        epsR[d + 1][I] = e[I] + c1 * Na[I];
        depsR[d + 1][I] = dR[I];
        e[I] = e[I] - c2 * Na[I];
      }
    }
    Sub<T, S> res;
    int nup;
    const int ph0 = lf_phase(f.w);
    S z[6], g;
    if (pair) {
      const int4 f2 = __ldg(t.lf + l + 1);
      const int ph1 = lf_phase(f2.w);
      S sL[6], sR[6];
      LeafTan<T> DL, DR;
      load_z_slot<S>(P, lf_slot(f.w), z);
      leaf_iso<T, S>(t.ph[ph0], e, z, sL, &DL, nullptr, gap_min ? &g : nullptr);
      if (gap_min) *gap_min = fmin(*gap_min, g);
      load_z_slot<S>(P, lf_slot(f2.w), z);
      leaf_iso<T, S>(t.ph[ph1], epsR[d], z, sR, &DR, nullptr, gap_min ? &g : nullptr);
      if (gap_min) *gap_min = fmin(*gap_min, g);
      const int node = __ldg(t.post + ipost++);
      S nd[3];
      T nt[3];
      load_ns<T, S>(P, node, nd, nt);
      T* gp = STORE ? gh.q + (size_t)(21 * node) * gh.s : nullptr;
      condense_bottom<T, STORE, S>(nd, nt, PassIn<S>::c1(t, node), PassIn<S>::c2(t, node), PassIn<S>::sc(t, node),
                                   node_c<T>(t, node), sL, DL, sR, DR, res, gp, gh.s, r2, t.ph[ph0].kind == 0,
                                   t.ph[ph1].kind == 0);
      --d;
      nup = f2.z - 1;
      l += 2;
    } else {
      S sg[6];
      LeafTan<T> D;
      load_z_slot<S>(P, lf_slot(f.w), z);
      leaf_iso<T, S>(t.ph[ph0], e, z, sg, &D, nullptr, gap_min ? &g : nullptr);
      if (gap_min) *gap_min = fmin(*gap_min, g);
      leaf_sub<T, S>(D, sg, res);
      nup = f.z;
      l += 1;
    }
    for (int u = 0; u < nup; ++u) {
      const int node = __ldg(t.post + ipost++);
      S nd[3];
      T nt[3];
      load_ns<T, S>(P, node, nd, nt);
      T* gp = STORE ? gh.q + (size_t)(21 * node) * gh.s : nullptr;
      const Sub<T, S> B = res;
      condense<T, STORE, S>(nd, nt, PassIn<S>::c1(t, node), PassIn<S>::c2(t, node), PassIn<S>::sc(t, node),
                            node_c<T>(t, node), pend[d], B, res, gp, gh.s, r2);
      --d;
    }
    if (d == 0) root = res;
    else pend[d] = res;
  }
}

// write_leaf_states for a compressed tree (tables of TreeDev).
__device__ inline void write_leaf_states_c(const TreeDev& t, const double Eloc[6], const PointArrays& P, double* zout,
                                           size_t zos, bool nan_out) {
  double epsR[KMAX + 1][6];
  int ipre = 0;
  for (int l = 0; l < t.Lc; ++l) {
    const int4 f = __ldg(t.lf + l);
    int d = f.x;
    double e[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) e[I] = (l == 0) ? Eloc[I] : epsR[d][I];
    for (int s = 0; s < f.y; ++s, ++d) {
      const int node = __ldg(t.pre + ipre++);
      const double nd[3] = {P.nrm[(3 * node) * P.ns], P.nrm[(3 * node + 1) * P.ns], P.nrm[(3 * node + 2) * P.ns]};
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double* ap = P.a + (size_t)(3 * node) * P.as;
      const double a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
      double Na[6];
      N_apply<double>(nd, ndr, a, Na);
#pragma unroll
      for (int I = 0; I < 6; ++I) { epsR[d + 1][I] = e[I] + c1 * Na[I]; e[I] -= c2 * Na[I]; }
    }
    const int slot = lf_slot(f.w);
    if (slot < 0) continue;
    double z[6], zn[6], sig[6];
    load_z_slot(P, slot, z);
    leaf_iso<double>(t.ph[lf_phase(f.w)], e, z, sig, nullptr, zn, nullptr);
    double* b = zout + (size_t)(6 * slot) * zos;
#pragma unroll
    for (int c = 0; c < 6; ++c) b[c * zos] = nan_out ? __longlong_as_double(0x7ff8000000000000LL) : zn[c];
  }
}

// Leaf strains from the jumps (top-down) and the return mapping at the final
// iterate: writes z^{n+1} of the inelastic leaves.
__device__ inline void write_leaf_states(const TreeDev& t, const double Eloc[6], const PointArrays& P, double* zout,
                                         size_t zos, bool nan_out) {
  const int K = t.K;
  double epsR[KMAX + 1][6];
  const int nbottom = 1 << (K - 1);
  for (int m = 0; m < nbottom; ++m) {
    const int top = (m == 0) ? 1 : K - __ffs(m) + 1;
    double e[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) e[I] = (m == 0) ? Eloc[I] : epsR[top][I];
    double eL[6], eR[6];
    for (int lvl = top; lvl <= K; ++lvl) {
      const int node = (1 << (lvl - 1)) + (m >> (K - lvl)) - 1;
      const double nd[3] = {P.nrm[(3 * node) * P.ns], P.nrm[(3 * node + 1) * P.ns], P.nrm[(3 * node + 2) * P.ns]};
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double* ap = P.a + (size_t)(3 * jump_index(P, K, lvl, node)) * P.as;
      const double a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
      double Na[6];
      N_apply<double>(nd, ndr, a, Na);
#pragma unroll
      for (int I = 0; I < 6; ++I) { eL[I] = e[I] - c2 * Na[I]; eR[I] = e[I] + c1 * Na[I]; }
      if (lvl < K) {
#pragma unroll
        for (int I = 0; I < 6; ++I) { epsR[lvl + 1][I] = eR[I]; e[I] = eL[I]; }
      }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      if (t.ph[side].kind == 0) continue;
      const int leaf = 2 * m + side;
      double z[6], zn[6], sig[6];
      load_z(t, P, leaf, side, z);
      leaf_iso<double>(t.ph[side], side ? eR : eL, z, sig, nullptr, zn, nullptr);
      const int slot = t.z_both ? leaf : (leaf >> 1);
      double* b = zout + (size_t)(6 * slot) * zos;
#pragma unroll
      for (int c = 0; c < 6; ++c) b[c * zos] = nan_out ? __longlong_as_double(0x7ff8000000000000LL) : zn[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint of the converged update (implicit function theorem, applied to the
// Euler-Lagrange equation R(a, theta) = A^T W sigma = 0 of Sec. 3.2).
//
// For a loss with gradient g = dL/d sigma_bar (local frame) the parameter
// gradient is dL/dtheta = d/dtheta [g . sigma_bar + mu . R] at fixed a = a* and
// fixed mu, where mu = (da/dE) g is the jump response to a macro strain
// perturbation g: the top-down map of the condensation, mu_j = H_j d_eps_j with
// d_eps_root = g (no extra solve; J is symmetric).  Writing g_i = g + (A mu)_i
// for the leaf strain perturbations and tau = average of D_i g_i over a
// subtree, the lagrangian is sum_i w_i g_i . sigma_i and its partial
// derivatives are
//   laminate normal: W c1 c2 [N(a)^T (tau_R - tau_L) + N(mu)^T (sb_R - sb_L)]
//                    (N(n) a = N(a) n), chained to the angles alpha, beta;
//   volume fractions through the subtree weights: with
//     Gam_X = (N mu)^T sb_X + (N a)^T tau_X,  Xi = (W_R Gam_R + W_L Gam_L) / W^2,
//   d/dW_L = W_R Xi, d/dW_R = -W_L Xi, and W_X is the sum of the leaf weights
//   below; leaf weight w_i directly: g_i . sigma_i.
struct AdjWork {
  const double* H; size_t hs;   // g, H of every laminate at a* (as stored by a Newton pass): [(21*node+c)*hs]
  double* mu;                   // [3*node + c] jump response, stride ws
  double* xi;                   // [node] weight term Xi, stride ws
  double* direct;               // [leaf] g_i . sigma_i, stride ws
  double* gab;                  // [node] dL/dalpha, [N + node] dL/dbeta, stride ws
  size_t ws;
};

// angles of laminate `node` from the point's shape-function values ph[m * phs] (the kernels pass the
// work array's copy in global memory)
__device__ __forceinline__ void node_angles(const TreeDev& t, int node, const double* ph, size_t phs, double& al,
                                            double& be) {
  al = 0.0; be = 0.0;
  for (int m = 0; m < t.M; ++m) {
    al += __ldg(t.p + node * t.M + m) * ph[m * phs];
    be += __ldg(t.q + node * t.M + m) * ph[m * phs];
  }
}

static __device__ void adjoint_pass(const TreeDev& t, const double Eloc[6], const double gl[6], const double* ph, size_t phs,
                             const PointArrays& P, const AdjWork& Wk) {
  const int K = t.K;
  double epsR[KMAX + 1][6], gR[KMAX + 1][6];
  double pend_s[KMAX + 1][6], pend_t[KMAX + 1][6];
  const int nbottom = 1 << (K - 1);
  const size_t ws = Wk.ws;
  for (int m = 0; m < nbottom; ++m) {
    const int top = (m == 0) ? 1 : K - __ffs(m) + 1;
    double e[6], ge[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      e[I] = (m == 0) ? Eloc[I] : epsR[top][I];
      ge[I] = (m == 0) ? gl[I] : gR[top][I];
    }
    double eL[6], eR[6], gL[6], gRr[6];
    for (int lvl = top; lvl <= K; ++lvl) {
      const int node = (1 << (lvl - 1)) + (m >> (K - lvl)) - 1;
      double nd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) nd[c] = P.nrm[(3 * node + c) * P.ns];
      const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double* ap = P.a + (size_t)(3 * jump_index(P, K, lvl, node)) * P.as;
      const double a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      const double* Hp = Wk.H + (size_t)(21 * node + 3) * Wk.hs;   // c1 c2 H, as the pass stores it
      const double ic = __ldg(t.ic12 + node);
      double mu[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
#pragma unroll
        for (int I = 0; I < 6; ++I) v += Hp[(6 * c + I) * Wk.hs] * ge[I];
        v *= ic;
        mu[c] = v;
        Wk.mu[(size_t)(3 * node + c) * ws] = v;
      }
      double Na[6], Nm[6];
      N_apply<double>(nd, ndr, a, Na);
      N_apply<double>(nd, ndr, mu, Nm);
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        eL[I] = e[I] - c2 * Na[I]; eR[I] = e[I] + c1 * Na[I];
        gL[I] = ge[I] - c2 * Nm[I]; gRr[I] = ge[I] + c1 * Nm[I];
      }
      if (lvl < K) {
#pragma unroll
        for (int I = 0; I < 6; ++I) { epsR[lvl + 1][I] = eR[I]; gR[lvl + 1][I] = gRr[I]; e[I] = eL[I]; ge[I] = gL[I]; }
      }
    }
    // leaves: stress, D g_i, direct weight term
    double sb[6], tb[6], sbL[6], tbL[6];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int leaf = 2 * m + side;
      double z[6], sig[6];
      LeafTan<double> D;
      load_z(t, P, leaf, side, z);
      leaf_iso<double>(t.ph[side], side ? eR : eL, z, sig, &D, nullptr, nullptr);
      const double* gi = side ? gRr : gL;
      const double tr = gi[0] + gi[1] + gi[2];
      double mg = 0.0, gs = 0.0;
#pragma unroll
      for (int I = 0; I < 6; ++I) { mg += D.m[I] * gi[I]; gs += gi[I] * sig[I]; }
      double tv[6];
#pragma unroll
      for (int I = 0; I < 6; ++I) tv[I] = 2.0 * D.mu * gi[I] - D.c * mg * D.m[I] + (I < 3 ? D.lam * tr : 0.0);
      Wk.direct[(size_t)leaf * ws] = gs;
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        if (side) { sb[I] = sig[I]; tb[I] = tv[I]; } else { sbL[I] = sig[I]; tbL[I] = tv[I]; }
      }
    }
    // laminates upwards while the finished one is a right child
    int lvl = K, idx = m;
    for (;;) {
      const int node = (1 << (lvl - 1)) + idx - 1;
      double nd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) nd[c] = P.nrm[(3 * node + c) * P.ns];
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double W = __ldg(t.sc + node) / (c1 * c2);
      const double* ap = P.a + (size_t)(3 * jump_index(P, K, lvl, node)) * P.as;
      const double a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      double mu[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) mu[c] = Wk.mu[(size_t)(3 * node + c) * ws];
      const double ar[3] = {a[0] * RS2, a[1] * RS2, a[2] * RS2}, mr[3] = {mu[0] * RS2, mu[1] * RS2, mu[2] * RS2};
      double ds[6], dt[6];
#pragma unroll
      for (int I = 0; I < 6; ++I) { ds[I] = sb[I] - sbL[I]; dt[I] = tb[I] - tbL[I]; }
      double u1[3], u2[3];
      Nt_apply<double>(a, ar, dt, u1);    // N(a)^T (tau_R - tau_L)
      Nt_apply<double>(mu, mr, ds, u2);   // N(mu)^T (sb_R - sb_L)
      const double sc = W * c1 * c2;
      const double gn[3] = {sc * (u1[0] + u2[0]), sc * (u1[1] + u2[1]), sc * (u1[2] + u2[2])};
      double al, be, sa, ca, sbeta, cbeta;
      node_angles(t, node, ph, phs, al, be);
      sincos(al, &sa, &ca);
      sincos(be, &sbeta, &cbeta);
      Wk.gab[(size_t)node * ws] = gn[0] * ca * cbeta + gn[1] * ca * sbeta - gn[2] * sa;
      Wk.gab[(size_t)(t.N + node) * ws] = -gn[0] * sa * sbeta + gn[1] * sa * cbeta;
      // weight terms: Gam_X = (N mu)^T sb_X + (N a)^T tau_X
      const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
      double Nm[6], Na[6];
      N_apply<double>(nd, ndr, mu, Nm);
      N_apply<double>(nd, ndr, a, Na);
      double GL = 0.0, GR = 0.0;
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        GL += Nm[I] * sbL[I] + Na[I] * tbL[I];
        GR += Nm[I] * sb[I] + Na[I] * tb[I];
      }
      const double WL = c1 * W, WR = c2 * W;
      Wk.xi[(size_t)node * ws] = (WR * GR + WL * GL) / (W * W);
      double so[6], to[6];
#pragma unroll
      for (int I = 0; I < 6; ++I) { so[I] = c1 * sbL[I] + c2 * sb[I]; to[I] = c1 * tbL[I] + c2 * tb[I]; }
      if (lvl == 1) break;
      if (!(idx & 1)) {
#pragma unroll
        for (int I = 0; I < 6; ++I) { pend_s[lvl][I] = so[I]; pend_t[lvl][I] = to[I]; }
        break;
      }
#pragma unroll
      for (int I = 0; I < 6; ++I) { sb[I] = so[I]; tb[I] = to[I]; sbL[I] = pend_s[lvl][I]; tbL[I] = pend_t[lvl][I]; }
      idx >>= 1;
      --lvl;
    }
  }
}

// Leaf-weight gradient: each leaf collects the direct term and, from every
// laminate above it, +W_R Xi (left subtree) or -W_L Xi (right subtree); then the
// normalisation w~ = w / S is undone: dL/dw_k = (G_k - sum_l G_l w~_l) / S.
static __device__ void adjoint_weights(const TreeDev& t, const double* wl, double S, const AdjWork& Wk, double* gw,
                                size_t gws) {
  const int K = t.K, L = t.L;
  const size_t ws = Wk.ws;
  double accR[KMAX + 2];
  double sum_gw = 0.0;
  const int nbottom = 1 << (K - 1);
  for (int m = 0; m < nbottom; ++m) {
    const int top = (m == 0) ? 1 : K - __ffs(m) + 1;
    double acc = (m == 0) ? 0.0 : accR[top];
    double aL = 0.0, aR = 0.0;
    for (int lvl = top; lvl <= K; ++lvl) {
      const int node = (1 << (lvl - 1)) + (m >> (K - lvl)) - 1;
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double W = __ldg(t.sc + node) / (c1 * c2);
      const double xi = Wk.xi[(size_t)node * ws];
      aL = acc + c2 * W * xi;   // left subtree: + W_R Xi
      aR = acc - c1 * W * xi;   // right subtree: - W_L Xi
      if (lvl < K) { accR[lvl + 1] = aR; acc = aL; }
    }
    const double G0 = Wk.direct[(size_t)(2 * m) * ws] + aL;
    const double G1 = Wk.direct[(size_t)(2 * m + 1) * ws] + aR;
    gw[(size_t)(2 * m) * gws] = G0;
    gw[(size_t)(2 * m + 1) * gws] = G1;
    sum_gw += G0 * __ldg(wl + 2 * m) + G1 * __ldg(wl + 2 * m + 1);
  }
  for (int l = 0; l < L; ++l) gw[(size_t)l * gws] = (gw[(size_t)l * gws] - sum_gw) / S;
}

// adjoint_pass over a compressed tree (tables of TreeDev): the same per-laminate and
// per-leaf terms, leaves one at a time, laminates numbered as in the state.
static __device__ void adjoint_pass_c(const TreeDev& t, const double Eloc[6], const double gl[6], const double* ph,
                               size_t phs, const PointArrays& P, const AdjWork& Wk) {
  double epsR[KMAX + 1][6], gR[KMAX + 1][6];
  double pend_s[KMAX + 1][6], pend_t[KMAX + 1][6];
  const size_t ws = Wk.ws;
  int ipre = 0, ipost = 0;
  for (int l = 0; l < t.Lc; ++l) {
    const int4 f = __ldg(t.lf + l);
    int d = f.x;
    double e[6], ge[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      e[I] = (l == 0) ? Eloc[I] : epsR[d][I];
      ge[I] = (l == 0) ? gl[I] : gR[d][I];
    }
    for (int s = 0; s < f.y; ++s, ++d) {
      const int node = __ldg(t.pre + ipre++);
      double nd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) nd[c] = P.nrm[(3 * node + c) * P.ns];
      const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double* ap = P.a + (size_t)(3 * node) * P.as;
      const double a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      const double* Hp = Wk.H + (size_t)(21 * node + 3) * Wk.hs;   // c1 c2 H, as the pass stores it
      const double ic = __ldg(t.ic12 + node);
      double mu[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double v = 0.0;
#pragma unroll
        for (int I = 0; I < 6; ++I) v += Hp[(6 * c + I) * Wk.hs] * ge[I];
        v *= ic;
        mu[c] = v;
        Wk.mu[(size_t)(3 * node + c) * ws] = v;
      }
      double Na[6], Nm[6];
      N_apply<double>(nd, ndr, a, Na);
      N_apply<double>(nd, ndr, mu, Nm);
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        epsR[d + 1][I] = e[I] + c1 * Na[I];
        gR[d + 1][I] = ge[I] + c1 * Nm[I];
        e[I] -= c2 * Na[I];
        ge[I] -= c2 * Nm[I];
      }
    }
    // the leaf: stress, D g_i, direct weight term
    double sb[6], tb[6];
    {
      double z[6];
      LeafTan<double> D;
      load_z_slot(P, lf_slot(f.w), z);
      leaf_iso<double>(t.ph[lf_phase(f.w)], e, z, sb, &D, nullptr, nullptr);
      const double tr = ge[0] + ge[1] + ge[2];
      double mg = 0.0, gs = 0.0;
#pragma unroll
      for (int I = 0; I < 6; ++I) { mg += D.m[I] * ge[I]; gs += ge[I] * sb[I]; }
#pragma unroll
      for (int I = 0; I < 6; ++I) tb[I] = 2.0 * D.mu * ge[I] - D.c * mg * D.m[I] + (I < 3 ? D.lam * tr : 0.0);
      Wk.direct[(size_t)lf_leaf(f.w) * ws] = gs;
    }
    // laminates completed by this leaf: left sibling pending at the same depth
    for (int u = 0; u < f.z; ++u) {
      const int node = __ldg(t.post + ipost++);
      double sbL[6], tbL[6];
#pragma unroll
      for (int I = 0; I < 6; ++I) { sbL[I] = pend_s[d][I]; tbL[I] = pend_t[d][I]; }
      double nd[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) nd[c] = P.nrm[(3 * node + c) * P.ns];
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double W = __ldg(t.sc + node) / (c1 * c2);
      const double* ap = P.a + (size_t)(3 * node) * P.as;
      const double a[3] = {ap[0], ap[P.as], ap[2 * P.as]};
      double mu[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) mu[c] = Wk.mu[(size_t)(3 * node + c) * ws];
      const double ar[3] = {a[0] * RS2, a[1] * RS2, a[2] * RS2}, mr[3] = {mu[0] * RS2, mu[1] * RS2, mu[2] * RS2};
      double ds[6], dt[6];
#pragma unroll
      for (int I = 0; I < 6; ++I) { ds[I] = sb[I] - sbL[I]; dt[I] = tb[I] - tbL[I]; }
      double u1[3], u2[3];
      Nt_apply<double>(a, ar, dt, u1);    // N(a)^T (tau_R - tau_L)
      Nt_apply<double>(mu, mr, ds, u2);   // N(mu)^T (sb_R - sb_L)
      const double sc = W * c1 * c2;
      const double gn[3] = {sc * (u1[0] + u2[0]), sc * (u1[1] + u2[1]), sc * (u1[2] + u2[2])};
      double al, be, sa, ca, sbeta, cbeta;
      node_angles(t, node, ph, phs, al, be);
      sincos(al, &sa, &ca);
      sincos(be, &sbeta, &cbeta);
      Wk.gab[(size_t)node * ws] = gn[0] * ca * cbeta + gn[1] * ca * sbeta - gn[2] * sa;
      Wk.gab[(size_t)(t.N + node) * ws] = -gn[0] * sa * sbeta + gn[1] * sa * cbeta;
      const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
      double Nm[6], Na[6];
      N_apply<double>(nd, ndr, mu, Nm);
      N_apply<double>(nd, ndr, a, Na);
      double GL = 0.0, GR = 0.0;
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        GL += Nm[I] * sbL[I] + Na[I] * tbL[I];
        GR += Nm[I] * sb[I] + Na[I] * tb[I];
      }
      const double WL = c1 * W, WR = c2 * W;
      Wk.xi[(size_t)node * ws] = (WR * GR + WL * GL) / (W * W);
#pragma unroll
      for (int I = 0; I < 6; ++I) { sb[I] = c1 * sbL[I] + c2 * sb[I]; tb[I] = c1 * tbL[I] + c2 * tb[I]; }
      --d;
    }
    if (d > 0) {
#pragma unroll
      for (int I = 0; I < 6; ++I) { pend_s[d][I] = sb[I]; pend_t[d][I] = tb[I]; }
    }
  }
}

// adjoint_weights over a compressed tree.  Leaves of weight zero get no gradient: the
// compressed tree holds nothing of them, and the weights' Macaulay bracket (Sec. 3.1)
// passes none below zero.
static __device__ void adjoint_weights_c(const TreeDev& t, const double* wl, double S, const AdjWork& Wk, double* gw,
                                  size_t gws) {
  const size_t ws = Wk.ws;
  double accR[KMAX + 2];
  double sum_gw = 0.0;
  for (int l = 0; l < t.L; ++l) gw[(size_t)l * gws] = 0.0;
  int ipre = 0;
  for (int l = 0; l < t.Lc; ++l) {
    const int4 f = __ldg(t.lf + l);
    int d = f.x;
    double acc = (l == 0) ? 0.0 : accR[d];
    for (int s = 0; s < f.y; ++s, ++d) {
      const int node = __ldg(t.pre + ipre++);
      const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
      const double W = __ldg(t.sc + node) / (c1 * c2);
      const double xi = Wk.xi[(size_t)node * ws];
      accR[d + 1] = acc - c1 * W * xi;   // right subtree: - W_L Xi
      acc += c2 * W * xi;                // left subtree: + W_R Xi
    }
    const int leaf = lf_leaf(f.w);
    const double G = Wk.direct[(size_t)leaf * ws] + acc;
    gw[(size_t)leaf * gws] = G;
    sum_gw += G * __ldg(wl + leaf);
  }
  for (int l = 0; l < t.Lc; ++l) {
    const int leaf = lf_leaf(__ldg(t.lf + l).w);
    gw[(size_t)leaf * gws] = (gw[(size_t)leaf * gws] - sum_gw) / S;
  }
}

// ---------------------------------------------------------------------------
// Tangent seeds of the adjoint, for trees of elastic phases.  With constant
// leaf tangents the DMN's tangent is the laminate recursion of Sec. 3.1 (Eq. of
// the stiffness propagation), here in the form of the condensation: a laminate
// with children tangents C_L, C_R (fractions c1, c2, normal n) has
//   Ch = c2 C_L + c1 C_R, dC = C_R - C_L, B = dC N, Kn = N^T Ch N, Y = Kn^-1 B^T,
//   C  = c1 C_L + c2 C_R - c1 c2 B Y.
// Reverse mode, for a symmetric Gb = dL/dC (dL = sum over all 36 entries of Gb dC):
//   Bb = -2 c1 c2 Gb Y^T,   Kb = c1 c2 Y Gb Y^T,
//   dL/dC_L = sym(c1 Gb + c2 N Kb N^T - Bb N^T),  dL/dC_R = sym(c2 Gb + c1 N Kb N^T + Bb N^T),
//   dL/dN   = 2 Ch N Kb + dC Bb,
//   dL/dc1  = Gb : (C_L - C_R) - (c2 - c1) Gb : (B Y) + Kb : (N^T B)   (c2 = 1 - c1).
// Matrices are full 6x6 here; packed arguments hold the upper triangle (sidx).

__device__ __forceinline__ void unpack_sym6(const double p[21], double A[6][6]) {
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = 0; J < 6; ++J) A[I][J] = p[sidx(I, J)];
}

__device__ __forceinline__ void n_matrix(const double n[3], double Nm[6][3]) {
  const double nr[3] = {n[0] * RS2, n[1] * RS2, n[2] * RS2};
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int j = 0; j < 3; ++j) Nm[I][j] = N_nonzero(I, j) ? N_entry<double>(n, nr, I, j) : 0.0;
}

// the laminate's tangent C (packed) from its children's
static __device__ void lam_tangent(const double n[3], double c1, double c2, const double CL[21], const double CR[21],
                            double C[21]) {
  double Nm[6][3];
  n_matrix(n, Nm);
  double ChN[6][3], B[6][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int P = 0; P < 6; ++P) {
        const int s2 = sidx(I, P);
        a += (c2 * CL[s2] + c1 * CR[s2]) * Nm[P][j];
        b += (CR[s2] - CL[s2]) * Nm[P][j];
      }
      ChN[I][j] = a; B[I][j] = b;
    }
  double K[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double v = 0.0;
#pragma unroll
      for (int P = 0; P < 6; ++P) v += Nm[P][i] * ChN[P][j];
      K[i][j] = v;
    }
  double Ki[3][3];
  inv3_sym<double>(K[0][0], 0.5 * (K[0][1] + K[1][0]), 0.5 * (K[0][2] + K[2][0]), K[1][1],
                   0.5 * (K[1][2] + K[2][1]), K[2][2], Ki);
  double Y[3][6];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int J = 0; J < 6; ++J) Y[m][J] = Ki[m][0] * B[J][0] + Ki[m][1] * B[J][1] + Ki[m][2] * B[J][2];
  const double c12 = c1 * c2;
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = I; J < 6; ++J) {
      const int s2 = sidx(I, J);
      C[s2] = c1 * CL[s2] + c2 * CR[s2] - c12 * (B[I][0] * Y[0][J] + B[I][1] * Y[1][J] + B[I][2] * Y[2][J]);
    }
}

static __device__ void lam_tangent_adjoint(const double n[3], double c1, double c2, const double CL[21], const double CR[21],
                                    const double Gbp[21], double GL[21], double GR[21], double nb[3], double& c1b) {
  double Nm[6][3];
  n_matrix(n, Nm);
  double Ch[6][6], dC[6][6], Gb[6][6];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = 0; J < 6; ++J) {
      const int s2 = sidx(I, J);
      Ch[I][J] = c2 * CL[s2] + c1 * CR[s2];
      dC[I][J] = CR[s2] - CL[s2];
      Gb[I][J] = Gbp[s2];
    }
  double ChN[6][3], B[6][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int P = 0; P < 6; ++P) { a += Ch[I][P] * Nm[P][j]; b += dC[I][P] * Nm[P][j]; }
      ChN[I][j] = a; B[I][j] = b;
    }
  double K[3][3], NB[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double v = 0.0, w = 0.0;
#pragma unroll
      for (int P = 0; P < 6; ++P) { v += Nm[P][i] * ChN[P][j]; w += Nm[P][i] * B[P][j]; }
      K[i][j] = v; NB[i][j] = w;
    }
  double Ki[3][3];
  inv3_sym<double>(K[0][0], 0.5 * (K[0][1] + K[1][0]), 0.5 * (K[0][2] + K[2][0]), K[1][1],
                   0.5 * (K[1][2] + K[2][1]), K[2][2], Ki);
  double Y[3][6];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int J = 0; J < 6; ++J) Y[m][J] = Ki[m][0] * B[J][0] + Ki[m][1] * B[J][1] + Ki[m][2] * B[J][2];
  const double c12 = c1 * c2;
  // T = Gb Y^T (6x3); Bb = -2 c12 T; Kb = c12 Y T
  double T[6][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      double v = 0.0;
#pragma unroll
      for (int J = 0; J < 6; ++J) v += Gb[I][J] * Y[m][J];
      T[I][m] = v;
    }
  double Bb[6][3], Kb[3][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int m = 0; m < 3; ++m) Bb[I][m] = -2.0 * c12 * T[I][m];
#pragma unroll
  for (int m = 0; m < 3; ++m)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = 0.0;
#pragma unroll
      for (int I = 0; I < 6; ++I) v += Y[m][I] * T[I][k];
      Kb[m][k] = c12 * v;
    }
  // dL/dc1
  double gLR = 0.0, gBY = 0.0, kNB = 0.0;
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = 0; J < 6; ++J) gLR -= Gb[I][J] * dC[I][J];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int m = 0; m < 3; ++m) gBY += B[I][m] * T[I][m];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) kNB += Kb[i][j] * NB[i][j];
  c1b = gLR - (c2 - c1) * gBY + kNB;
  // N Kb N^T and Bb N^T
  double NK[6][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int k = 0; k < 3; ++k) NK[I][k] = Nm[I][0] * Kb[0][k] + Nm[I][1] * Kb[1][k] + Nm[I][2] * Kb[2][k];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = I; J < 6; ++J) {
      const double nkn = NK[I][0] * Nm[J][0] + NK[I][1] * Nm[J][1] + NK[I][2] * Nm[J][2];
      const double bn = 0.5 * (Bb[I][0] * Nm[J][0] + Bb[I][1] * Nm[J][1] + Bb[I][2] * Nm[J][2]
                               + Bb[J][0] * Nm[I][0] + Bb[J][1] * Nm[I][1] + Bb[J][2] * Nm[I][2]);
      const int s2 = sidx(I, J);
      GL[s2] = c1 * Gb[I][J] + c2 * nkn - bn;
      GR[s2] = c2 * Gb[I][J] + c1 * nkn + bn;
    }
  // dL/dN = 2 Ch N Kb + dC Bb, then dL/dn through N's entries
  double Nb[6][3];
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double v = 2.0 * (ChN[I][0] * Kb[0][k] + ChN[I][1] * Kb[1][k] + ChN[I][2] * Kb[2][k]);
#pragma unroll
      for (int P = 0; P < 6; ++P) v += dC[I][P] * Bb[P][k];
      Nb[I][k] = v;
    }
  nb[0] = Nb[0][0]; nb[1] = Nb[1][1]; nb[2] = Nb[2][2];
  // shear rows: N[I][a] = n_b / sqrt2, N[I][b] = n_a / sqrt2 for the index pair (a, b) of row I
#pragma unroll
  for (int I = 3; I < 6; ++I) {
    const int a = I == 3 ? 1 : 0, b = I == 5 ? 1 : 2;
    nb[b] += RS2 * Nb[I][a];
    nb[a] += RS2 * Nb[I][b];
  }
}

// children of a laminate: >= 0 a laminate (array index), -1 - phase a leaf
__device__ __forceinline__ void lam_kids(const TreeDev& t, bool cmp, int node, int& k1, int& k2) {
  if (cmp) {
    k1 = __ldg(t.kid + 2 * node);
    k2 = __ldg(t.kid + 2 * node + 1);
  } else if (node >= (1 << (t.K - 1)) - 1) {   // bottom laminate: leaves of phases 0 and 1
    k1 = -1; k2 = -2;
  } else {
    k1 = 2 * node + 1; k2 = 2 * node + 2;
  }
}

// The tangent's adjoint of one point, level by level of the full tree's heap positions, so
// that the lanes of a warp share a level: lane `lane` of `nl` takes every nl-th position of the
// level (the laminate standing there, if any; compressed trees skip passed-through and dead
// positions).  A laminate's children stand at deeper positions, so the forward pass (the
// children's stiffnesses to the laminate's, stored in Cst [21 N]) runs from level K up, and the
// reverse pass (the laminate's adjoint, read from Gst [21 N], to its children's adjoints, its
// normal's and its volume fraction's) from the root down; the caller orders the levels (a warp
// barrier between them).  Cph: the leaf stiffnesses of the two phases; ph[m * phs]: the point's
// shape-function values; strides Wk.ws.
__device__ __forceinline__ int heap_to_lam(const TreeDev& t, int h) { return t.hcid ? __ldg(t.hcid + h) : h; }

__device__ __forceinline__ void phase_stiffnesses(const TreeDev& t, double Cph[2][21]) {
#pragma unroll
  for (int f = 0; f < 2; ++f)
#pragma unroll
    for (int I = 0; I < 6; ++I)
#pragma unroll
      for (int J = I; J < 6; ++J)
        Cph[f][sidx(I, J)] = ((I < 3 && J < 3) ? t.ph[f].lam : 0.0) + (I == J ? 2.0 * t.ph[f].G : 0.0);
}

static __device__ void tangent_level_fwd(const TreeDev& t, bool cmp, int lvl, int lane, int nl, const PointArrays& P,
                                  const double Cph[2][21], double* Cst, size_t ws) {
  const int h0 = (1 << (lvl - 1)) - 1, nh = 1 << (lvl - 1);
  for (int x = lane; x < nh; x += nl) {
    const int node = heap_to_lam(t, h0 + x);
    if (node < 0) continue;
    int k1, k2;
    lam_kids(t, cmp, node, k1, k2);
    double CL[21], CR[21], C[21], nd[3];
#pragma unroll
    for (int k = 0; k < 21; ++k) {
      CL[k] = k1 >= 0 ? Cst[(size_t)(21 * k1 + k) * ws] : Cph[-1 - k1][k];
      CR[k] = k2 >= 0 ? Cst[(size_t)(21 * k2 + k) * ws] : Cph[-1 - k2][k];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) nd[c] = P.nrm[(3 * node + c) * P.ns];
    lam_tangent(nd, __ldg(t.c1 + node), __ldg(t.c2 + node), CL, CR, C);
#pragma unroll
    for (int k = 0; k < 21; ++k) Cst[(size_t)(21 * node + k) * ws] = C[k];
  }
}

static __device__ void tangent_level_rev(const TreeDev& t, bool cmp, int lvl, int lane, int nl, const double* ph, size_t phs,
                                  const PointArrays& P, const double Cph[2][21], const double* Cst, double* Gst,
                                  const AdjWork& Wk) {
  const size_t ws = Wk.ws;
  const int h0 = (1 << (lvl - 1)) - 1, nh = 1 << (lvl - 1);
  for (int x = lane; x < nh; x += nl) {
    const int node = heap_to_lam(t, h0 + x);
    if (node < 0) continue;
    int k1, k2;
    lam_kids(t, cmp, node, k1, k2);
    double CL[21], CR[21], G[21], GL[21], GR[21], nd[3], nb[3], c1b;
#pragma unroll
    for (int k = 0; k < 21; ++k) {
      CL[k] = k1 >= 0 ? Cst[(size_t)(21 * k1 + k) * ws] : Cph[-1 - k1][k];
      CR[k] = k2 >= 0 ? Cst[(size_t)(21 * k2 + k) * ws] : Cph[-1 - k2][k];
      G[k] = Gst[(size_t)(21 * node + k) * ws];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) nd[c] = P.nrm[(3 * node + c) * P.ns];
    const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
    lam_tangent_adjoint(nd, c1, c2, CL, CR, G, GL, GR, nb, c1b);
    double al, be, sa, ca, sbeta, cbeta;
    node_angles(t, node, ph, phs, al, be);
    sincos(al, &sa, &ca);
    sincos(be, &sbeta, &cbeta);
    Wk.gab[(size_t)node * ws] += nb[0] * ca * cbeta + nb[1] * ca * sbeta - nb[2] * sa;
    Wk.gab[(size_t)(t.N + node) * ws] += -nb[0] * sa * sbeta + nb[1] * sa * cbeta;
    const double W = __ldg(t.sc + node) / (c1 * c2);
    Wk.xi[(size_t)node * ws] += c1b / (W * W);   // c1 = W_L / W: d/dW_L = W_R Xi, d/dW_R = -W_L Xi
    if (k1 >= 0)
#pragma unroll
      for (int k = 0; k < 21; ++k) Gst[(size_t)(21 * k1 + k) * ws] = GL[k];
    if (k2 >= 0)
#pragma unroll
      for (int k = 0; k < 21; ++k) Gst[(size_t)(21 * k2 + k) * ws] = GR[k];
  }
}

// the laminate at the root: the whole tree's root, or the topmost one kept by compression
__device__ __forceinline__ int tangent_root(const TreeDev& t, bool cmp) { return cmp ? t.N - 1 : 0; }

// ---------------------------------------------------------------------------
// One Newton pass of one point by a group of lanes of a warp (32, 16 or 8 lanes: one, two or four
// points per warp), level by level of a heap tree (small batches, where one point per thread
// leaves most of the GPU idle).  The per-laminate arithmetic is that of tree_pass -- the same
// functions in the same order -- so a point's iterates are those of the thread-per-point kernel
// to rounding (the two are compiled apart, and the residual's squares are summed in another
// order: the lanes' partial sums are reduced at the end).  The lanes share a level's laminates:
// top-down the jump correction and the children's strains (each laminate hands them to its
// children through ein / dein), then at the bottom level the leaves and the structured
// condensation, then bottom-up the condensation of each level from its children's results
// (sb, dc); a barrier of the group separates the levels.  Fewer lanes per point leave fewer
// lanes idle on the upper levels (at depth 8 levels 1-5 hold 31 laminates) at the price of more
// points in flight.
// Per-point arrays (one block per group), field-major over the laminates, stride N (the
// handle's largest tree): jumps a [N][3]; c1 c2 (g, H) [21][N]; ein [6][N] (FP64) and dein [6][N]
// (T); results sb [6][N] (FP64), ds and C [27][N] (T); normals in P (nrm / nrmf [N][3], stride 1);
// compressed trees also le [6][N] (FP64).
template <typename T>
struct WarpSlot {
  const double* a_in; double* a_out;
  const T* gh_in; T* gh_out;
  double* ein; T* dein;
  double* sb; T* dc;
  int N;
  double* le;   // compressed trees: the strain of a laminate's leaf child beside a laminate child [6][N]
};

template <typename T>
__device__ __forceinline__ void warp_sub_store(const WarpSlot<T>& W, int node, const Sub<T>& r) {
#pragma unroll
  for (int I = 0; I < 6; ++I) W.sb[I * W.N + node] = r.sb[I];
#pragma unroll
  for (int I = 0; I < 6; ++I) W.dc[I * W.N + node] = r.ds[I];
#pragma unroll
  for (int k = 0; k < 21; ++k) W.dc[(6 + k) * W.N + node] = r.C[k];
}
template <typename T>
__device__ __forceinline__ void warp_sub_load(const WarpSlot<T>& W, int node, Sub<T>& r) {
#pragma unroll
  for (int I = 0; I < 6; ++I) r.sb[I] = W.sb[I * W.N + node];
#pragma unroll
  for (int I = 0; I < 6; ++I) r.ds[I] = W.dc[I * W.N + node];
#pragma unroll
  for (int k = 0; k < 21; ++k) r.C[k] = W.dc[(6 + k) * W.N + node];
}

// One level of the descent (lvl = 1 .. K): lane `lane` of the point's `lanes` lanes takes every
// lanes-th laminate of the level; at the bottom level it also evaluates the laminate's leaves and
// its structured condensation.  Adds the lane's share of the squared residual norm to r2.
template <typename T>
__device__ void warp_descend_level(const TreeDev& t, const double Eloc[6], const PointArrays& P, const WarpSlot<T>& W,
                                   bool apply, T step, int lvl, int lane, int lanes, double& r2) {
  const int K = t.K, NS = W.N;
  const int h0 = (1 << (lvl - 1)) - 1, nh = 1 << (lvl - 1);
  for (int x = lane; x < nh; x += lanes) {
    const int node = h0 + x;
    double e[6];
    T de[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      e[I] = lvl == 1 ? Eloc[I] : W.ein[I * NS + node];
      de[I] = lvl == 1 ? (T)0 : W.dein[I * NS + node];
    }
    double nd[3];
    T nt[3];
    load_n<T>(P, node, nd, nt);
    const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
    double a[3] = {W.a_in[3 * node], W.a_in[3 * node + 1], W.a_in[3 * node + 2]};
    T da[3] = {(T)0, (T)0, (T)0};
    {
      const T* gp = W.gh_in + node;
      const T ic = ic12_of<T>(t, node);   // the stored step is c1 c2 (g, H)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T v = step * gp[c * NS];
#pragma unroll
        for (int I = 0; I < 6; ++I) v += gp[(3 + 6 * c + I) * NS] * de[I];
        da[c] = apply ? v * ic : (T)0;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) { a[c] += widen(da[c]); W.a_out[3 * node + c] = a[c]; }
    }
    const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
    double Na[6], eL[6], eR[6];
    N_apply<double>(nd, ndr, a, Na);
#pragma unroll
    for (int I = 0; I < 6; ++I) { eL[I] = e[I] - c2 * Na[I]; eR[I] = e[I] + c1 * Na[I]; }
    if (lvl < K) {
      const NodeC<T> cc = node_c<T>(t, node);
      const T ntr[3] = {nt[0] * (T)RS2, nt[1] * (T)RS2, nt[2] * (T)RS2};
      T Nda[6], dR[6];
      N_apply<T>(nt, ntr, da, Nda);
#pragma unroll
      for (int I = 0; I < 6; ++I) { dR[I] = de[I] + cc.c1 * Nda[I]; de[I] = de[I] - cc.c2 * Nda[I]; }
      const int k1 = 2 * node + 1, k2 = 2 * node + 2;
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        W.ein[I * NS + k1] = eL[I]; W.dein[I * NS + k1] = de[I];
        W.ein[I * NS + k2] = eR[I]; W.dein[I * NS + k2] = dR[I];
      }
    } else {   // the bottom laminate's two leaves and its structured condensation
      double z[6], sL[6], sR[6];
      LeafTan<T> DL, DR;
      load_z<double>(t, P, 2 * x, 0, z);
      leaf_iso<T, double>(t.ph[0], eL, z, sL, &DL, nullptr, nullptr);
      load_z<double>(t, P, 2 * x + 1, 1, z);
      leaf_iso<T, double>(t.ph[1], eR, z, sR, &DR, nullptr, nullptr);
      Sub<T> res;
      condense_bottom<T, true, double>(nd, nt, c1, c2, __ldg(t.sc + node), node_c<T>(t, node), sL, DL, sR, DR, res,
                                       W.gh_out + node, (size_t)NS, r2, t.ph[0].kind == 0, t.ph[1].kind == 0);
      warp_sub_store<T>(W, node, res);
    }
  }
}

// One level of the condensation above the bottom one (lvl = K - 1 .. 1), from the children's results.
template <typename T>
__device__ void warp_condense_level(const TreeDev& t, const PointArrays& P, const WarpSlot<T>& W, int lvl, int lane,
                                    int lanes, double& r2) {
  const int h0 = (1 << (lvl - 1)) - 1, nh = 1 << (lvl - 1);
  for (int x = lane; x < nh; x += lanes) {
    const int node = h0 + x;
    double nd[3];
    T nt[3];
    load_n<T>(P, node, nd, nt);
    Sub<T> L, R, res;
    warp_sub_load<T>(W, 2 * node + 1, L);
    warp_sub_load<T>(W, 2 * node + 2, R);
    condense<T, true, double>(nd, nt, __ldg(t.c1 + node), __ldg(t.c2 + node), __ldg(t.sc + node), node_c<T>(t, node),
                              L, R, res, W.gh_out + node, (size_t)W.N, r2);
    warp_sub_store<T>(W, node, res);
  }
}

// Compressed trees (the tables of TreeDev): the same pass level by level of the full tree's heap
// positions.  A kept laminate keeps its heap position; its children (kid) may stand several levels
// deeper, or be leaves.  A laminate whose children are two leaves condenses them on the way down
// (structured condensation); a leaf beside a laminate is evaluated when its parent condenses, from
// the strain the parent handed it (le).  The root is the last laminate.
template <typename T>
__device__ void warp_descend_level_c(const TreeDev& t, const double Eloc[6], const PointArrays& P,
                                     const WarpSlot<T>& W, bool apply, T step, int lvl, int lane, int lanes,
                                     double& r2) {
  const int NS = W.N, root = t.N - 1;
  const int h0 = (1 << (lvl - 1)) - 1, nh = 1 << (lvl - 1);
  for (int x = lane; x < nh; x += lanes) {
    const int node = __ldg(t.hcid + h0 + x);
    if (node < 0) continue;
    double e[6];
    T de[6];
#pragma unroll
    for (int I = 0; I < 6; ++I) {
      e[I] = node == root ? Eloc[I] : W.ein[I * NS + node];
      de[I] = node == root ? (T)0 : W.dein[I * NS + node];
    }
    double nd[3];
    T nt[3];
    load_n<T>(P, node, nd, nt);
    const double c1 = __ldg(t.c1 + node), c2 = __ldg(t.c2 + node);
    double a[3] = {W.a_in[3 * node], W.a_in[3 * node + 1], W.a_in[3 * node + 2]};
    T da[3] = {(T)0, (T)0, (T)0};
    {
      const T* gp = W.gh_in + node;
      const T ic = ic12_of<T>(t, node);   // the stored step is c1 c2 (g, H)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        T v = step * gp[c * NS];
#pragma unroll
        for (int I = 0; I < 6; ++I) v += gp[(3 + 6 * c + I) * NS] * de[I];
        da[c] = apply ? v * ic : (T)0;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) { a[c] += widen(da[c]); W.a_out[3 * node + c] = a[c]; }
    }
    const double ndr[3] = {nd[0] * RS2, nd[1] * RS2, nd[2] * RS2};
    double Na[6], eL[6], eR[6];
    N_apply<double>(nd, ndr, a, Na);
#pragma unroll
    for (int I = 0; I < 6; ++I) { eL[I] = e[I] - c2 * Na[I]; eR[I] = e[I] + c1 * Na[I]; }
    const int k1 = __ldg(t.kid + 2 * node), k2 = __ldg(t.kid + 2 * node + 1);
    if (k1 >= 0 || k2 >= 0) {   // a laminate child: hand the strains and their corrections down
      const NodeC<T> cc = node_c<T>(t, node);
      const T ntr[3] = {nt[0] * (T)RS2, nt[1] * (T)RS2, nt[2] * (T)RS2};
      T Nda[6], dR[6];
      N_apply<T>(nt, ntr, da, Nda);
#pragma unroll
      for (int I = 0; I < 6; ++I) { dR[I] = de[I] + cc.c1 * Nda[I]; de[I] = de[I] - cc.c2 * Nda[I]; }
#pragma unroll
      for (int I = 0; I < 6; ++I) {
        if (k1 >= 0) { W.ein[I * NS + k1] = eL[I]; W.dein[I * NS + k1] = de[I]; }
        else W.le[I * NS + node] = eL[I];
        if (k2 >= 0) { W.ein[I * NS + k2] = eR[I]; W.dein[I * NS + k2] = dR[I]; }
        else W.le[I * NS + node] = eR[I];
      }
    } else {   // two leaves and their structured condensation
      const int p1 = -1 - k1, p2 = -1 - k2;
      double z[6], sL[6], sR[6];
      LeafTan<T> DL, DR;
      load_z_slot<double>(P, __ldg(t.kslot + 2 * node), z);
      leaf_iso<T, double>(t.ph[p1], eL, z, sL, &DL, nullptr, nullptr);
      load_z_slot<double>(P, __ldg(t.kslot + 2 * node + 1), z);
      leaf_iso<T, double>(t.ph[p2], eR, z, sR, &DR, nullptr, nullptr);
      Sub<T> res;
      condense_bottom<T, true, double>(nd, nt, c1, c2, __ldg(t.sc + node), node_c<T>(t, node), sL, DL, sR, DR, res,
                                       W.gh_out + node, (size_t)NS, r2, t.ph[p1].kind == 0, t.ph[p2].kind == 0);
      warp_sub_store<T>(W, node, res);
    }
  }
}

// the subtree result of laminate `node`'s child on `side`: a laminate's from W, or the leaf's
// (evaluated at the strain in le)
template <typename T>
__device__ __forceinline__ void warp_child_c(const TreeDev& t, const PointArrays& P, const WarpSlot<T>& W, int node,
                                             int side, Sub<T>& r) {
  const int k = __ldg(t.kid + 2 * node + side);
  if (k >= 0) {
    warp_sub_load<T>(W, k, r);
    return;
  }
  double e[6], z[6], sg[6];
#pragma unroll
  for (int I = 0; I < 6; ++I) e[I] = W.le[I * W.N + node];
  LeafTan<T> D;
  load_z_slot<double>(P, __ldg(t.kslot + 2 * node + side), z);
  leaf_iso<T, double>(t.ph[-1 - k], e, z, sg, &D, nullptr, nullptr);
  leaf_sub<T, double>(D, sg, r);
}

template <typename T>
__device__ void warp_condense_level_c(const TreeDev& t, const PointArrays& P, const WarpSlot<T>& W, int lvl,
                                      int lane, int lanes, double& r2) {
  const int h0 = (1 << (lvl - 1)) - 1, nh = 1 << (lvl - 1);
  for (int x = lane; x < nh; x += lanes) {
    const int node = __ldg(t.hcid + h0 + x);
    if (node < 0 || (__ldg(t.kid + 2 * node) < 0 && __ldg(t.kid + 2 * node + 1) < 0)) continue;
    double nd[3];
    T nt[3];
    load_n<T>(P, node, nd, nt);
    Sub<T> L, R, res;
    warp_child_c<T>(t, P, W, node, 0, L);
    warp_child_c<T>(t, P, W, node, 1, R);
    condense<T, true, double>(nd, nt, __ldg(t.c1 + node), __ldg(t.c2 + node), __ldg(t.sc + node), node_c<T>(t, node),
                              L, R, res, W.gh_out + node, (size_t)W.N, r2);
    warp_sub_store<T>(W, node, res);
  }
}

// The whole pass for the point of a group of `lanes` lanes (gmask: the group's lanes in the warp):
// levels in order, a barrier of the group between them.  Returns this lane's share of the squared
// residual norm; the root's result is at node 0 of W (heap trees) or at its last laminate (CMP).
template <typename T, bool CMP>
__device__ double warp_tree_pass(const TreeDev& t, const double Eloc[6], const PointArrays& P, const WarpSlot<T>& W,
                                 bool apply, T step, int lane, int lanes, unsigned gmask) {
  double r2 = 0.0;
  for (int lvl = 1; lvl <= t.K; ++lvl) {
    if (CMP) warp_descend_level_c<T>(t, Eloc, P, W, apply, step, lvl, lane, lanes, r2);
    else warp_descend_level<T>(t, Eloc, P, W, apply, step, lvl, lane, lanes, r2);
    __syncwarp(gmask);
  }
  for (int lvl = t.K - 1; lvl >= 1; --lvl) {
    if (CMP) warp_condense_level_c<T>(t, P, W, lvl, lane, lanes, r2);
    else warp_condense_level<T>(t, P, W, lvl, lane, lanes, r2);
    __syncwarp(gmask);
  }
  return r2;
}

// ---------------------------------------------------------------------------
// Mandel rotation R_IJ = (w_I w_J / 2)(Q_ia Q_jb + Q_ib Q_ja) for index pairs
// I = (i, j), J = (a, b), w = 1 (normal) or sqrt 2 (shear): sigma_glob =
// R sigma_loc, E_loc = R^T E_glob, C_glob = R C_loc R^T.
__device__ __forceinline__ void mandel_rotation(const double Q[9], double R[6][6]) {
  const int pi[6] = {0, 1, 2, 1, 0, 0}, pj[6] = {0, 1, 2, 2, 2, 1};
#pragma unroll
  for (int I = 0; I < 6; ++I)
#pragma unroll
    for (int J = 0; J < 6; ++J) {
      const int i = pi[I], j = pj[I], a = pi[J], b = pj[J];
      const double wIJ = ((I < 3) ? 1.0 : 1.41421356237309504880) * ((J < 3) ? 1.0 : 1.41421356237309504880) * 0.5;
      R[I][J] = wIJ * (Q[3 * i + a] * Q[3 * j + b] + Q[3 * i + b] * Q[3 * j + a]);
    }
}

}  // namespace dmn
