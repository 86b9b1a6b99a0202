// FP64 CPU oracle for differentiable depth-sorted Gaussian-splat rasterization.
//
// TEST INFRASTRUCTURE ONLY.  This file is the plain, slow definition that the
// CUDA path is checked against.  Only tests, the smoke check and the benchmark's
// CPU-baseline leg may load it.  It shares no code, header or constant table
// with the CUDA library, and it never reads anything the CUDA path produced.
//
// What it computes (paper: "Efficient Differentiable Hardware Rasterization for
// 3D Gaussian Splatting", arXiv 2505.18764):
//   * Sec. 2.1.1, Eq. 1: a splat is (mu_3D, o, SH colour, Sigma_3D = R S S^T R^T).
//   * Sec. 2.1.2: mu_2D = proj(W mu_3D), Sigma_2D = J W Sigma_3D W^T J^T (+ 0.3 I
//     low-pass dilation, EWA splatting, the reference the paper cites).
//   * Sec. 2.1.2, Eq. 2: front-to-back compositing C = sum_i T_i alpha_i c_i,
//     T_i = prod_{k<i} (1 - alpha_k); fragments with alpha < 1/255 skipped.
//   * Sec. 2.1.4 / Procedure 1: T-culling, a fragment is skipped iff T_i < t_cull.
//   * Eq. 3 and Eq. 4: dL/dc_i = dL/dC alpha_i T_i and
//     dL/dalpha_i = dL/dC (c_i T_i - sum_{k>i} T_k alpha_k c_k / (1 - alpha_i)),
//     written out with explicit suffix sums (the plain definition), not with the
//     front-to-back recurrence of Eq. 5-7 that the fast path uses.
//   * Chain rule from (c_i, alpha_i) to the 3D parameters ("bwd_diff" in
//     Procedure 1), written with explicit small-matrix loops.
//
// Readings where the paper is silent (each listed in the design notes):
//   * alpha = min(0.99, o exp(power)); derivative of the clamp is 0 above 0.99.
//   * near-plane cull t_z <= znear (0.2); splats with |q| = 0 are invalid.
//   * real orthonormal SH basis with the Condon-Shortley phase, index l^2+l+m,
//     colour = max(0, sum sh Y + 0.5), additionally min(1, .) under unorm formats.
//   * depth order: ascending camera-space z, ties broken by splat index.
//   * background colour 0.
//
// Parity unpinned: relation to the paper's own images/gradients (no weights or
// code are available).  Every function below is pinned by tests (closed forms,
// invariants, library special functions, finite differences, brute force).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double kAlphaMin = 1.0 / 255.0;   // Sec. 2.1.2 (8-bit colour threshold)
constexpr double kAlphaMax = 0.99;          // reading: opacity clamp
constexpr double kDilation = 0.3;           // reading: EWA low-pass filter

struct Camera {
  double R[3][3];
  double t[3];
  double campos[3];
  double fx, fy, cx, cy;
  int W, H;
  double znear;
};

Camera read_camera(const double* c) {
  Camera cam;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) cam.R[i][j] = c[i * 4 + j];
    cam.t[i] = c[i * 4 + 3];
  }
  for (int i = 0; i < 3; ++i) cam.campos[i] = c[12 + i];
  cam.fx = c[15];
  cam.fy = c[16];
  cam.cx = c[17];
  cam.cy = c[18];
  cam.W = static_cast<int>(c[19]);
  cam.H = static_cast<int>(c[20]);
  cam.znear = c[21];
  return cam;
}

// Options passed as a flat double array.
struct Opts {
  double t_cull;      // skip fragment iff T_i < t_cull (0 disables)
  int clamp01;        // colour additionally saturated to [0, 1] (unorm formats)
  int quant;          // 0 none, 1 fp16, 2 unorm16, 3 unorm8 (state rounding emulation)
  int per_fragment;   // 1: round (C, T) after every fragment (render-target blending)
  double band_cut;    // tie band on |power - ln(1/(255 o))|
  double band_depth;  // tie band on relative depth difference of consecutive fragments
  double band_t;      // tie band on |T - t_cull| / t_cull
  double band_near;   // tie band on |t_z - znear|
  double band_clamp;  // tie band on |o exp(power) - 0.99|
};

Opts read_opts(const double* o) {
  Opts p;
  p.t_cull = o[0];
  p.clamp01 = static_cast<int>(o[1]);
  p.quant = static_cast<int>(o[2]);
  p.per_fragment = static_cast<int>(o[3]);
  p.band_cut = o[4];
  p.band_depth = o[5];
  p.band_t = o[6];
  p.band_near = o[7];
  p.band_clamp = o[8];
  return p;
}

// ---------------------------------------------------------------------------
// Reduced-precision rounding (Sec. 3.3 state formats), round-to-nearest-even.
// ---------------------------------------------------------------------------
double round_half_even(double x) { return std::nearbyint(x); }  // default FE_TONEAREST

double to_fp16(double x) {
  if (x == 0.0 || !std::isfinite(x)) return x;
  double ax = std::fabs(x);
  if (ax >= 65520.0) return std::copysign(INFINITY, x);
  int e;
  std::frexp(ax, &e);                      // ax = m * 2^e, m in [0.5, 1)
  int exp_unbiased = e - 1;                // ax = 1.f * 2^exp_unbiased
  if (exp_unbiased < -14) exp_unbiased = -14;  // subnormal range: fixed quantum 2^-24
  double quantum = std::ldexp(1.0, exp_unbiased - 10);
  double r = round_half_even(ax / quantum) * quantum;
  return std::copysign(r, x);
}

double to_unorm(double x, int bits) {
  double s = std::ldexp(1.0, bits) - 1.0;
  double c = std::min(1.0, std::max(0.0, x));
  return round_half_even(c * s) / s;
}

double quantize(double x, int mode) {
  switch (mode) {
    case 1: return to_fp16(x);
    case 2: return to_unorm(x, 16);
    case 3: return to_unorm(x, 8);
    default: return x;
  }
}

// ---------------------------------------------------------------------------
// Real spherical harmonics with the Condon-Shortley phase.
//   P_l(z) = 2^-l sum_k (-1)^k C(l,k) C(2l-2k, l) z^(l-2k)          (Legendre)
//   P_l^m(z) = (-1)^m (1 - z^2)^(m/2) d^m P_l / dz^m                 (CS phase)
//   K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)
//   Y_{l,0} = K_l^0 P_l(z)
//   Y_{l,m>0} = sqrt(2) K_l^m P_l^m(z) cos(m phi)
//   Y_{l,m<0} = sqrt(2) K_l^|m| P_l^|m|(z) sin(|m| phi)
// On the unit sphere (1 - z^2)^(m/2) cos(m phi) = Re((x + i y)^m) and
// (1 - z^2)^(m/2) sin(m phi) = Im((x + i y)^m), which gives each Y as a
// polynomial in (x, y, z); its gradient is taken of that polynomial.
// ---------------------------------------------------------------------------
double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

double factorial(int n) {
  double r = 1.0;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// coefficients c[p] of z^p for d^m P_l / dz^m
std::vector<double> legendre_deriv_coeffs(int l, int m) {
  std::vector<double> c(l + 1, 0.0);
  for (int k = 0; 2 * k <= l; ++k) {
    int p = l - 2 * k;
    c[p] = std::ldexp(1.0, -l) * ((k % 2) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l);
  }
  for (int d = 0; d < m; ++d) {
    std::vector<double> n(l + 1, 0.0);
    for (int p = 1; p <= l; ++p) n[p - 1] = c[p] * p;
    c.swap(n);
  }
  return c;
}

double poly_eval(const std::vector<double>& c, double z) {
  double r = 0.0;
  for (int p = static_cast<int>(c.size()) - 1; p >= 0; --p) r = r * z + c[p];
  return r;
}

// Per (l, |m|): normalisation and the coefficients of d^m P_l / dz^m and of
// d^(m+1) P_l / dz^(m+1), built once from the formulas above.
struct ShTables {
  double K[4][4];
  std::vector<double> q[4][4], q1[4][4];
  ShTables() {
    for (int l = 0; l <= 3; ++l)
      for (int am = 0; am <= l; ++am) {
        K[l][am] = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * factorial(l - am) / factorial(l + am));
        q[l][am] = legendre_deriv_coeffs(l, am);
        q1[l][am] = legendre_deriv_coeffs(l, am + 1);
      }
  }
};

const ShTables& sh_tables() {
  static const ShTables t;  // thread-safe initialisation
  return t;
}

// Evaluates all (deg+1)^2 basis functions at a unit direction; optional gradient.
void sh_basis(int deg, const double dir[3], double* Y, double* dY /* [K][3] or null */) {
  const ShTables& tab = sh_tables();
  const double x = dir[0], y = dir[1], z = dir[2];
  for (int l = 0; l <= deg; ++l) {
    for (int m = -l; m <= l; ++m) {
      const int am = std::abs(m);
      const double K = tab.K[l][am];
      const double cs = (am % 2) ? -1.0 : 1.0;  // (-1)^m Condon-Shortley phase
      const double Q = poly_eval(tab.q[l][am], z);
      const double Qz = poly_eval(tab.q1[l][am], z);
      // w^m and w^(m-1) with w = x + i y
      double re = 1.0, im = 0.0, re1 = 0.0, im1 = 0.0;
      for (int k = 0; k < am; ++k) {
        re1 = re;
        im1 = im;
        const double nr = re * x - im * y;
        const double ni = re * y + im * x;
        re = nr;
        im = ni;
      }
      double A, Ax, Ay, scale;
      if (m == 0) {
        A = 1.0; Ax = 0.0; Ay = 0.0; scale = K;
      } else if (m > 0) {
        A = re; Ax = am * re1; Ay = -am * im1; scale = std::sqrt(2.0) * K * cs;
      } else {
        A = im; Ax = am * im1; Ay = am * re1; scale = std::sqrt(2.0) * K * cs;
      }
      const int idx = l * l + l + m;
      Y[idx] = scale * Q * A;
      if (dY) {
        dY[idx * 3 + 0] = scale * Q * Ax;
        dY[idx * 3 + 1] = scale * Q * Ay;
        dY[idx * 3 + 2] = scale * Qz * A;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Per-splat projection (Sec. 2.1.1 Eq. 1, Sec. 2.1.2).
// ---------------------------------------------------------------------------
struct Splat {
  bool valid = false;
  double qn[4], qnorm;
  double scale[3];
  double Rq[3][3];           // rotation of the normalised quaternion
  double M[3][3];            // R diag(s)
  double S3[3][3];           // Sigma_3D
  double t[3];               // camera-space centre
  double J[2][3];            // projection Jacobian at t
  double Tm[2][3];           // J W
  double S2[2][2];           // Sigma_2D (dilated)
  double conic[3];           // (a, b, c) of Sigma_2D^-1 = [[a, b], [b, c]]
  double mu2[2];
  double dir[3], vnorm;      // view direction (normalised) and |mu - campos|
  double Y[16], dY[48];
  double raw[3], rgb[3];
  double opacity;
  double depth;
};

void project_one(const double* mu, const double* s, const double* q, double o, const double* sh,
                 int deg, const Camera& cam, int clamp01, Splat& sp) {
  sp = Splat();
  sp.opacity = o;
  for (int i = 0; i < 3; ++i) sp.scale[i] = s[i];
  const double qq = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  sp.qnorm = std::sqrt(qq);
  for (int i = 0; i < 3; ++i) {
    sp.t[i] = cam.t[i];
    for (int j = 0; j < 3; ++j) sp.t[i] += cam.R[i][j] * mu[j];
  }
  sp.depth = sp.t[2];
  if (!(qq > 0.0) || !(sp.t[2] > cam.znear)) return;
  for (int i = 0; i < 4; ++i) sp.qn[i] = q[i] / sp.qnorm;
  const double w = sp.qn[0], x = sp.qn[1], y = sp.qn[2], z = sp.qn[3];
  double (&R)[3][3] = sp.Rq;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) sp.M[i][j] = R[i][j] * s[j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += sp.M[i][k] * sp.M[j][k];
      sp.S3[i][j] = a;
    }
  const double tx = sp.t[0], ty = sp.t[1], tz = sp.t[2];
  sp.J[0][0] = cam.fx / tz; sp.J[0][1] = 0.0;         sp.J[0][2] = -cam.fx * tx / (tz * tz);
  sp.J[1][0] = 0.0;         sp.J[1][1] = cam.fy / tz; sp.J[1][2] = -cam.fy * ty / (tz * tz);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += sp.J[i][k] * cam.R[k][j];
      sp.Tm[i][j] = a;
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) a += sp.Tm[i][k] * sp.S3[k][l] * sp.Tm[j][l];
      sp.S2[i][j] = a + (i == j ? kDilation : 0.0);
    }
  const double det = sp.S2[0][0] * sp.S2[1][1] - sp.S2[0][1] * sp.S2[1][0];
  if (!(det > 0.0)) return;
  sp.conic[0] = sp.S2[1][1] / det;
  sp.conic[1] = -sp.S2[0][1] / det;
  sp.conic[2] = sp.S2[0][0] / det;
  sp.mu2[0] = cam.fx * tx / tz + cam.cx;
  sp.mu2[1] = cam.fy * ty / tz + cam.cy;
  double v[3];
  for (int i = 0; i < 3; ++i) v[i] = mu[i] - cam.campos[i];
  sp.vnorm = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int i = 0; i < 3; ++i) sp.dir[i] = v[i] / sp.vnorm;
  const int K = (deg + 1) * (deg + 1);
  sh_basis(deg, sp.dir, sp.Y, sp.dY);
  for (int c = 0; c < 3; ++c) {
    double a = 0.5;
    for (int k = 0; k < K; ++k) a += sh[k * 3 + c] * sp.Y[k];
    sp.raw[c] = a;
    double r = std::max(0.0, a);
    if (clamp01) r = std::min(1.0, r);
    sp.rgb[c] = r;
  }
  sp.valid = true;
}

struct Scene {
  int N;
  const double* means;
  const double* scales;
  const double* quats;
  const double* opac;
  const double* sh;
  int deg;
};

void project_all(const Scene& sc, const Camera& cam, int clamp01, std::vector<Splat>& out) {
  out.resize(sc.N);
  const int K = (sc.deg + 1) * (sc.deg + 1);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < sc.N; ++i)
    project_one(sc.means + 3 * i, sc.scales + 3 * i, sc.quats + 4 * i, sc.opac[i],
                sc.sh + static_cast<size_t>(i) * K * 3, sc.deg, cam, clamp01, out[i]);
}

// Ascending depth, ties by index (std::stable_sort over index order).
std::vector<int> depth_order(const std::vector<Splat>& sp) {
  std::vector<int> ord;
  ord.reserve(sp.size());
  for (int i = 0; i < static_cast<int>(sp.size()); ++i)
    if (sp[i].valid) ord.push_back(i);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return sp[a].depth < sp[b].depth; });
  return ord;
}

// ---------------------------------------------------------------------------
// One pixel: the ordered fragment list (Eq. 2 with the 1/255 and T-cull rules).
// ---------------------------------------------------------------------------
struct Frag {
  int id;
  double dx, dy;     // pixel centre minus mu_2D
  double G;          // exp(power)
  double at;         // o * G (unclamped alpha)
  double alpha;      // min(0.99, at)
  double T;          // transmittance before this fragment
};

struct PixelResult {
  double C[3];
  double T;
  int nfrag;
  int last;          // splat index of the last fragment, -1 if none
  int ambig;         // bit 0 cutoff band, 1 depth tie, 2 T-cull band, 3 near plane, 4 clamp band
};

void trace_pixel(int px, int py, const std::vector<Splat>& sp, const std::vector<int>& ord,
                 const Camera& cam, const Opts& op, std::vector<Frag>* frags, PixelResult& res) {
  const double ux = px + 0.5, uy = py + 0.5;
  double C[3] = {0.0, 0.0, 0.0};
  double T = 1.0;
  res.nfrag = 0;
  res.last = -1;
  res.ambig = 0;
  double prev_depth = -1.0;
  bool culled = false;
  if (frags) frags->clear();
  for (int id : ord) {
    const Splat& s = sp[id];
    const double dx = ux - s.mu2[0], dy = uy - s.mu2[1];
    const double power = -0.5 * (s.conic[0] * dx * dx + 2.0 * s.conic[1] * dx * dy + s.conic[2] * dy * dy);
    const double G = std::exp(power);
    const double at = s.opacity * G;
    const double alpha = std::min(kAlphaMax, at);
    // tie bands: a decision that FP32 evaluation may take the other way
    if (s.opacity > 0.0 && std::fabs(power - std::log(1.0 / (255.0 * s.opacity))) < op.band_cut)
      res.ambig |= 1;
    if (alpha < kAlphaMin) continue;
    if (culled) continue;
    if (std::fabs(s.depth - cam.znear) < op.band_near) res.ambig |= 8;
    if (op.t_cull > 0.0 && std::fabs(T - op.t_cull) < op.band_t * op.t_cull) res.ambig |= 4;
    if (T < op.t_cull) {  // T-culling (Procedure 1); T never grows, so the rest are culled too
      culled = true;
      continue;
    }
    if (prev_depth >= 0.0 && std::fabs(s.depth - prev_depth) <= op.band_depth * std::fabs(s.depth))
      res.ambig |= 2;
    if (std::fabs(at - kAlphaMax) < op.band_clamp) res.ambig |= 16;
    prev_depth = s.depth;
    if (frags) frags->push_back(Frag{id, dx, dy, G, at, alpha, T});
    for (int c = 0; c < 3; ++c) {
      C[c] += T * alpha * s.rgb[c];
      if (op.per_fragment) C[c] = quantize(C[c], op.quant);
    }
    T *= (1.0 - alpha);
    if (op.per_fragment) T = quantize(T, op.quant);
    res.nfrag++;
    res.last = id;
  }
  for (int c = 0; c < 3; ++c) res.C[c] = C[c];
  res.T = T;
}

// 2D gradient accumulators per splat: mu2 (2), conic a b c (3), rgb (3), opacity (1).
constexpr int kG2 = 9;

// Per-pixel backward with Eq. 3 and Eq. 4 (explicit suffix sums) and the chain
// rule from (c_i, alpha_i) to the 2D splat parameters.  `Cprime1` optionally
// replaces C'_1 = sum_k T_k alpha_k c_k by a stored (rounded) colour.
void pixel_backward(const std::vector<Frag>& fr, const std::vector<Splat>& sp, const double g[3],
                    const double* Cprime1, double* acc /* [N][9] */) {
  const int n = static_cast<int>(fr.size());
  // contributions w_k = T_k alpha_k c_k and their suffix sums S_i = sum_{k>i} w_k
  std::vector<double> S((n + 1) * 3, 0.0);
  for (int i = n - 1; i >= 0; --i)
    for (int c = 0; c < 3; ++c)
      S[i * 3 + c] = S[(i + 1) * 3 + c] + fr[i].T * fr[i].alpha * sp[fr[i].id].rgb[c];
  double shift[3] = {0.0, 0.0, 0.0};
  if (Cprime1)
    for (int c = 0; c < 3; ++c) shift[c] = Cprime1[c] - S[c];
  for (int i = 0; i < n; ++i) {
    const Frag& f = fr[i];
    const Splat& s = sp[f.id];
    double* a = acc + static_cast<size_t>(f.id) * kG2;
    double dL_dalpha = 0.0;
    for (int c = 0; c < 3; ++c) {
      a[5 + c] += g[c] * f.alpha * f.T;                                   // Eq. 3
      const double tail = S[(i + 1) * 3 + c] + shift[c];
      dL_dalpha += g[c] * (s.rgb[c] * f.T - tail / (1.0 - f.alpha));      // Eq. 4
    }
    const double d_at = (f.at < kAlphaMax) ? dL_dalpha : 0.0;
    a[8] += f.G * d_at;                                // d/d opacity
    const double d_power = f.at * d_at;
    a[2] += -0.5 * f.dx * f.dx * d_power;              // conic a
    a[3] += -f.dx * f.dy * d_power;                    // conic b (off-diagonal, counted once)
    a[4] += -0.5 * f.dy * f.dy * d_power;              // conic c
    a[0] += (s.conic[0] * f.dx + s.conic[1] * f.dy) * d_power;   // mu_2D x
    a[1] += (s.conic[1] * f.dx + s.conic[2] * f.dy) * d_power;   // mu_2D y
  }
}

// Chain rule from the 2D gradients to the 3D parameters of one splat.
void splat_backward(const Splat& s, const double* g2, const double* sh, int deg, const Camera& cam,
                    int clamp01, double* gmu, double* gs, double* gq, double* go, double* gsh) {
  const int K = (deg + 1) * (deg + 1);
  for (int i = 0; i < 3; ++i) { gmu[i] = 0.0; gs[i] = 0.0; }
  for (int i = 0; i < 4; ++i) gq[i] = 0.0;
  *go = g2[8];
  for (int k = 0; k < K * 3; ++k) gsh[k] = 0.0;
  if (!s.valid) return;
  // colour: rgb = clamp(raw), raw = sum sh_k Y_k(dir) + 0.5
  double graw[3];
  for (int c = 0; c < 3; ++c) {
    const bool pass = s.raw[c] > 0.0 && (!clamp01 || s.raw[c] < 1.0);
    graw[c] = pass ? g2[5 + c] : 0.0;
  }
  double gdir[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k)
    for (int c = 0; c < 3; ++c) {
      gsh[k * 3 + c] = s.Y[k] * graw[c];
      for (int j = 0; j < 3; ++j) gdir[j] += sh[k * 3 + c] * graw[c] * s.dY[k * 3 + j];
    }
  double dd = 0.0;
  for (int j = 0; j < 3; ++j) dd += s.dir[j] * gdir[j];
  for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - s.dir[j] * dd) / s.vnorm;
  // conic -> Sigma_2D:  G_Sigma = -Q G_Q Q with G_Q = [[ga, gb/2], [gb/2, gc]]
  const double Q[2][2] = {{s.conic[0], s.conic[1]}, {s.conic[1], s.conic[2]}};
  const double GQ[2][2] = {{g2[2], 0.5 * g2[3]}, {0.5 * g2[3], g2[4]}};
  double tmp[2][2], GS2[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      tmp[i][j] = 0.0;
      for (int k = 0; k < 2; ++k) tmp[i][j] += Q[i][k] * GQ[k][j];
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      GS2[i][j] = 0.0;
      for (int k = 0; k < 2; ++k) GS2[i][j] -= tmp[i][k] * Q[k][j];
    }
  // Sigma_2D = Tm S3 Tm^T + 0.3 I:  G_S3 = Tm^T G_S2 Tm, G_Tm = 2 G_S2 Tm S3
  double GS3[3][3], GT[2][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l) a += s.Tm[k][i] * GS2[k][l] * s.Tm[l][j];
      GS3[i][j] = a;
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 3; ++l) a += GS2[i][k] * s.Tm[k][l] * s.S3[l][j];
      GT[i][j] = 2.0 * a;
    }
  // Tm = J W:  G_J = G_Tm W^T
  double GJ[2][3];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += GT[i][k] * cam.R[j][k];
      GJ[i][j] = a;
    }
  const double tx = s.t[0], ty = s.t[1], tz = s.t[2];
  const double fx = cam.fx, fy = cam.fy;
  double gt[3] = {0.0, 0.0, 0.0};
  // J(t)
  gt[0] += GJ[0][2] * (-fx / (tz * tz));
  gt[1] += GJ[1][2] * (-fy / (tz * tz));
  gt[2] += GJ[0][0] * (-fx / (tz * tz)) + GJ[0][2] * (2.0 * fx * tx / (tz * tz * tz)) +
           GJ[1][1] * (-fy / (tz * tz)) + GJ[1][2] * (2.0 * fy * ty / (tz * tz * tz));
  // mu_2D(t)
  gt[0] += g2[0] * fx / tz;
  gt[1] += g2[1] * fy / tz;
  gt[2] += -g2[0] * fx * tx / (tz * tz) - g2[1] * fy * ty / (tz * tz);
  // t = W mu + w
  for (int j = 0; j < 3; ++j)
    for (int i = 0; i < 3; ++i) gmu[j] += cam.R[i][j] * gt[i];
  // Sigma_3D = M M^T, M = R diag(s)
  double GM[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double a = 0.0;
      for (int k = 0; k < 3; ++k) a += GS3[i][k] * s.M[k][j];
      GM[i][j] = 2.0 * a;
    }
  // M_ij = R_ij s_j:  dL/ds_j = sum_i G_M_ij R_ij,  G_R_ij = G_M_ij s_j
  double GR[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      gs[j] += s.Rq[i][j] * GM[i][j];
      GR[i][j] = GM[i][j] * s.scale[j];
    }
  // R(q_hat): partial derivatives of each entry with respect to (w, x, y, z)
  const double w = s.qn[0], x = s.qn[1], y = s.qn[2], z = s.qn[3];
  const double dR[3][3][4] = {
      {{0, 0, -4 * y, -4 * z}, {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x}},
      {{2 * z, 2 * y, 2 * x, 2 * w}, {0, -4 * x, 0, -4 * z}, {-2 * x, -2 * w, 2 * z, 2 * y}},
      {{-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y}, {0, -4 * x, -4 * y, 0}}};
  double gqn[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 4; ++k) gqn[k] += GR[i][j] * dR[i][j][k];
  double qd = 0.0;
  for (int k = 0; k < 4; ++k) qd += s.qn[k] * gqn[k];
  for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - s.qn[k] * qd) / s.qnorm;
}

int num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int thread_id() {
#ifdef _OPENMP
  return omp_get_thread_num();
#else
  return 0;
#endif
}

}  // namespace

extern "C" {

int oracle_num_threads() { return num_threads(); }

// Threads the parallel loops use from now on (0 or less: all cores).
int oracle_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#endif
  return num_threads();
}

// Y[n][K] (and dY[n][K][3] if non-null) for unit directions dirs[n][3].
int oracle_sh_basis(int deg, const double* dirs, int n, double* Y, double* dY) {
  if (deg < 0 || deg > 3) return -1;
  const int K = (deg + 1) * (deg + 1);
  for (int i = 0; i < n; ++i) sh_basis(deg, dirs + 3 * i, Y + static_cast<size_t>(i) * K,
                                       dY ? dY + static_cast<size_t>(i) * K * 3 : nullptr);
  return 0;
}

// Per-splat projection.  out[N][20]:
//   0 valid, 1-2 mu_2D, 3-5 Sigma_2D (00, 01, 11), 6-8 conic (a, b, c), 9-11 rgb,
//   12 depth (t_z), 13-15 raw colour, 16-18 camera-space t, 19 unused.
int oracle_project(int N, const double* means, const double* scales, const double* quats,
                   const double* opac, const double* sh, int deg, const double* camv, int clamp01,
                   double* out) {
  if (deg < 0 || deg > 3 || N < 0) return -1;
  const Camera cam = read_camera(camv);
  Scene sc{N, means, scales, quats, opac, sh, deg};
  std::vector<Splat> sp;
  project_all(sc, cam, clamp01, sp);
  for (int i = 0; i < N; ++i) {
    double* o = out + static_cast<size_t>(i) * 20;
    std::memset(o, 0, 20 * sizeof(double));
    const Splat& s = sp[i];
    o[0] = s.valid ? 1.0 : 0.0;
    o[1] = s.mu2[0]; o[2] = s.mu2[1];
    o[3] = s.S2[0][0]; o[4] = s.S2[0][1]; o[5] = s.S2[1][1];
    o[6] = s.conic[0]; o[7] = s.conic[1]; o[8] = s.conic[2];
    for (int c = 0; c < 3; ++c) { o[9 + c] = s.rgb[c]; o[13 + c] = s.raw[c]; o[16 + c] = s.t[c]; }
    o[12] = s.depth;
  }
  return 0;
}

// Stable ascending sort of u32 keys; order[i] = index of the i-th smallest.
int oracle_stable_sort_u32(int n, const uint32_t* keys, int32_t* order) {
  std::vector<int32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return keys[a] < keys[b]; });
  std::copy(idx.begin(), idx.end(), order);
  return 0;
}

// Depth order of the valid splats; returns the count.
int oracle_depth_order(int N, const double* means, const double* scales, const double* quats,
                       const double* opac, const double* sh, int deg, const double* camv,
                       int32_t* order) {
  const Camera cam = read_camera(camv);
  Scene sc{N, means, scales, quats, opac, sh, deg};
  std::vector<Splat> sp;
  project_all(sc, cam, 0, sp);
  std::vector<int> ord = depth_order(sp);
  std::copy(ord.begin(), ord.end(), order);
  return static_cast<int>(ord.size());
}

// Forward render of the listed pixels (linear index y*W+x), or of all pixels if
// pixels == null.  color[npix][3], T[npix], nfrag[npix], last[npix], ambig[npix];
// any output pointer may be null.  timings (if non-null) receives the seconds
// spent in projection + depth order and in tracing.
int oracle_render(int N, const double* means, const double* scales, const double* quats,
                  const double* opac, const double* sh, int deg, const double* camv,
                  const double* optv, const int32_t* pixels, int npix, double* color, double* Tout,
                  int32_t* nfrag, int32_t* last, int32_t* ambig, double* timings) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const Camera cam = read_camera(camv);
  const Opts op = read_opts(optv);
  Scene sc{N, means, scales, quats, opac, sh, deg};
  std::vector<Splat> sp;
  project_all(sc, cam, op.clamp01, sp);
  const std::vector<int> ord = depth_order(sp);
  const auto t1 = clk::now();
  const int total = pixels ? npix : cam.W * cam.H;
#pragma omp parallel for schedule(dynamic, 1)
  for (int p = 0; p < total; ++p) {
    const int lin = pixels ? pixels[p] : p;
    PixelResult r;
    trace_pixel(lin % cam.W, lin / cam.W, sp, ord, cam, op, nullptr, r);
    double C[3] = {r.C[0], r.C[1], r.C[2]};
    double T = r.T;
    if (op.quant && !op.per_fragment) {  // store-only rounding of the saved state
      for (int c = 0; c < 3; ++c) C[c] = quantize(C[c], op.quant);
      T = quantize(T, op.quant);
    }
    if (color) for (int c = 0; c < 3; ++c) color[static_cast<size_t>(p) * 3 + c] = C[c];
    if (Tout) Tout[p] = T;
    if (nfrag) nfrag[p] = r.nfrag;
    if (last) last[p] = r.last;
    if (ambig) ambig[p] = r.ambig;
  }
  if (timings) {
    timings[0] = std::chrono::duration<double>(t1 - t0).count();
    timings[1] = std::chrono::duration<double>(clk::now() - t1).count();
  }
  return 0;
}

// Backward: dL/dC [H][W][3] -> parameter gradients (overwritten, not
// accumulated).  Optionally returns the image and the per-splat 2D gradients.
// quant_cprime: if nonzero, C'_1 is the stored colour rounded with opts.quant
// (emulates a reduced-precision saved state read back by the backward pass).
// pixels (linear y*W+x) restricts the traced pixels to a subset (null = all);
// the image is then written for the listed pixels only.  timings (if non-null)
// receives the seconds spent in projection + depth order and in tracing.
int oracle_backward(int N, const double* means, const double* scales, const double* quats,
                    const double* opac, const double* sh, int deg, const double* camv,
                    const double* optv, const double* dLdC, int quant_cprime, const int32_t* pixels,
                    int npix, double* image, double* g_means, double* g_scales, double* g_quats,
                    double* g_opac, double* g_sh, double* g2d_out, double* timings) {
  using clk = std::chrono::steady_clock;
  const auto t0 = clk::now();
  const Camera cam = read_camera(camv);
  const Opts op = read_opts(optv);
  Scene sc{N, means, scales, quats, opac, sh, deg};
  std::vector<Splat> sp;
  project_all(sc, cam, op.clamp01, sp);
  const std::vector<int> ord = depth_order(sp);
  const auto t1 = clk::now();
  const int nt = num_threads();
  std::vector<double> acc(static_cast<size_t>(nt) * N * kG2, 0.0);
  const int total = pixels ? npix : cam.W * cam.H;
#pragma omp parallel
  {
    std::vector<Frag> fr;
    double* mine = acc.data() + static_cast<size_t>(thread_id()) * N * kG2;
#pragma omp for schedule(dynamic, 1)
    for (int q = 0; q < total; ++q) {
      const int p = pixels ? pixels[q] : q;
      PixelResult r;
      trace_pixel(p % cam.W, p / cam.W, sp, ord, cam, op, &fr, r);
      if (image) for (int c = 0; c < 3; ++c) image[static_cast<size_t>(p) * 3 + c] = r.C[c];
      double cp[3];
      const double* cp1 = nullptr;
      if (quant_cprime && op.quant) {
        for (int c = 0; c < 3; ++c) cp[c] = quantize(r.C[c], op.quant);
        cp1 = cp;
      }
      pixel_backward(fr, sp, dLdC + static_cast<size_t>(p) * 3, cp1, mine);
    }
  }
  std::vector<double> g2(static_cast<size_t>(N) * kG2, 0.0);
  for (int t = 0; t < nt; ++t)
    for (size_t k = 0; k < g2.size(); ++k) g2[k] += acc[static_cast<size_t>(t) * N * kG2 + k];
  if (g2d_out) std::copy(g2.begin(), g2.end(), g2d_out);
  const int K = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < N; ++i)
    splat_backward(sp[i], g2.data() + static_cast<size_t>(i) * kG2, sh + static_cast<size_t>(i) * K * 3,
                   deg, cam, op.clamp01, g_means + 3 * i, g_scales + 3 * i, g_quats + 4 * i,
                   g_opac + i, g_sh + static_cast<size_t>(i) * K * 3);
  const auto t2 = clk::now();
  if (timings) {
    timings[0] = std::chrono::duration<double>(t1 - t0).count();
    timings[1] = std::chrono::duration<double>(t2 - t1).count();
  }
  return 0;
}

// Gradients of a few selected splats at full image size: only the pixels that
// can hold a fragment of a selected splat are traced (every pixel whose centre
// lies in the ellipse's bounding box, widened by one pixel).  Outputs are per
// selected splat: g2d[n][9], g_means[n][3], g_scales[n][3], g_quats[n][4],
// g_opac[n], g_sh[n][K][3]; pixel_count[n] = pixels traced for that splat.
int oracle_splat_grads(int N, const double* means, const double* scales, const double* quats,
                       const double* opac, const double* sh, int deg, const double* camv,
                       const double* optv, const double* dLdC, const int32_t* ids, int nids,
                       double* g2d_out, double* g_means, double* g_scales, double* g_quats,
                       double* g_opac, double* g_sh, int32_t* pixel_count) {
  const Camera cam = read_camera(camv);
  const Opts op = read_opts(optv);
  Scene sc{N, means, scales, quats, opac, sh, deg};
  std::vector<Splat> sp;
  project_all(sc, cam, op.clamp01, sp);
  const std::vector<int> ord = depth_order(sp);
  const int K = (deg + 1) * (deg + 1);
  for (int j = 0; j < nids; ++j) {
    const int id = ids[j];
    const Splat& s = sp[id];
    std::vector<double> g2(kG2, 0.0);
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    if (s.valid && s.opacity * 255.0 > 1.0) {
      // alpha >= 1/255 only where d^T Q d <= 2 ln(255 o); the box of that ellipse
      // has half-widths sqrt(k Sigma_00), sqrt(k Sigma_11).
      const double k = 2.0 * std::log(255.0 * s.opacity);
      const double ex = std::sqrt(k * s.S2[0][0]), ey = std::sqrt(k * s.S2[1][1]);
      x0 = std::max(0, static_cast<int>(std::floor(s.mu2[0] - ex - 0.5)) - 1);
      x1 = std::min(cam.W - 1, static_cast<int>(std::ceil(s.mu2[0] + ex - 0.5)) + 1);
      y0 = std::max(0, static_cast<int>(std::floor(s.mu2[1] - ey - 0.5)) - 1);
      y1 = std::min(cam.H - 1, static_cast<int>(std::ceil(s.mu2[1] + ey - 0.5)) + 1);
    }
    const int w = std::max(0, x1 - x0 + 1), h = std::max(0, y1 - y0 + 1);
    pixel_count[j] = w * h;
    // The splats (in depth order) that can reach a pixel of this rectangle.  A
    // splat has alpha >= 1/255 only inside the ellipse d^T Q d <= 2 ln(255 o)
    // (and its tie band only inside d^T Q d <= 2 (ln(255 o) + band_cut)); one
    // whose box of the wider ellipse, grown by a pixel, misses the rectangle's
    // pixel centres adds nothing there, so tracing the rest gives the same
    // fragment lists as tracing every splat.
    std::vector<int> sub;
    if (w > 0 && h > 0) {
      const double rx0 = x0 + 0.5, rx1 = x1 + 0.5, ry0 = y0 + 0.5, ry1 = y1 + 0.5;
      for (int id2 : ord) {
        const Splat& t = sp[id2];
        const double kk = 2.0 * (std::log(255.0 * t.opacity) + op.band_cut);
        if (!(t.opacity > 0.0) || !(kk >= 0.0)) continue;
        const double ex2 = std::sqrt(kk * t.S2[0][0]) + 1.0, ey2 = std::sqrt(kk * t.S2[1][1]) + 1.0;
        if (t.mu2[0] + ex2 < rx0 || t.mu2[0] - ex2 > rx1 || t.mu2[1] + ey2 < ry0 ||
            t.mu2[1] - ey2 > ry1)
          continue;
        sub.push_back(id2);
      }
    }
    const int nt = num_threads();
    std::vector<double> part(static_cast<size_t>(nt) * kG2, 0.0);
#pragma omp parallel
    {
      std::vector<Frag> fr;
      std::vector<double> local(kG2, 0.0);
#pragma omp for schedule(dynamic, 4)
      for (int p = 0; p < w * h; ++p) {
        const int px = x0 + p % w, py = y0 + p / w;
        PixelResult r;
        trace_pixel(px, py, sp, sub, cam, op, &fr, r);
        const int n = static_cast<int>(fr.size());
        // suffix sums over the whole fragment list, then keep the selected splat
        std::vector<double> S((n + 1) * 3, 0.0);
        for (int i = n - 1; i >= 0; --i)
          for (int c = 0; c < 3; ++c)
            S[i * 3 + c] = S[(i + 1) * 3 + c] + fr[i].T * fr[i].alpha * sp[fr[i].id].rgb[c];
        const double* g = dLdC + (static_cast<size_t>(py) * cam.W + px) * 3;
        for (int i = 0; i < n; ++i) {
          if (fr[i].id != id) continue;
          const Frag& f = fr[i];
          double dL_dalpha = 0.0;
          for (int c = 0; c < 3; ++c) {
            local[5 + c] += g[c] * f.alpha * f.T;
            dL_dalpha += g[c] * (s.rgb[c] * f.T - S[(i + 1) * 3 + c] / (1.0 - f.alpha));
          }
          const double d_at = (f.at < kAlphaMax) ? dL_dalpha : 0.0;
          local[8] += f.G * d_at;
          const double d_power = f.at * d_at;
          local[2] += -0.5 * f.dx * f.dx * d_power;
          local[3] += -f.dx * f.dy * d_power;
          local[4] += -0.5 * f.dy * f.dy * d_power;
          local[0] += (s.conic[0] * f.dx + s.conic[1] * f.dy) * d_power;
          local[1] += (s.conic[1] * f.dx + s.conic[2] * f.dy) * d_power;
        }
      }
      for (int k = 0; k < kG2; ++k) part[static_cast<size_t>(thread_id()) * kG2 + k] = local[k];
    }
    for (int t = 0; t < nt; ++t)
      for (int k = 0; k < kG2; ++k) g2[k] += part[static_cast<size_t>(t) * kG2 + k];
    for (int k = 0; k < kG2; ++k) g2d_out[static_cast<size_t>(j) * kG2 + k] = g2[k];
    splat_backward(s, g2.data(), sh + static_cast<size_t>(id) * K * 3, deg, cam, op.clamp01,
                   g_means + 3 * j, g_scales + 3 * j, g_quats + 4 * j, g_opac + j,
                   g_sh + static_cast<size_t>(j) * K * 3);
  }
  return 0;
}

}  // extern "C"
