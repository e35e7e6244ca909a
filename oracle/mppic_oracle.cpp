// MP-PIC parcel-grid coupling step: plain, slow FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may load this file:
// only the test suite, the package smoke check and the benchmark's CPU-baseline
// leg use it. It shares no code, header or constant with the CUDA library.
//
// It restates the parcel side of the multiphase particle-in-cell model of
// Woo et al., "Development of an Equation-based Parallelization Method for
// Multiphase Particle-in-Cell Simulations" (arXiv 2211.15605):
//   * parcel volume V = w * V_particle                       (Sec. 2.1)
//   * dx_P/dt = u_P                                          (Eq. 3)
//   * eps_P rho_P du_P/dt = -eps_P grad p + F_P + eps_P rho_P g - grad tau_P
//                                                            (Eq. 4)
//   * tau_P = p_s eps_P^beta / max[eps_CP - eps_P, alpha (1 - eps_P)]
//                                                            (Eq. 5)
//   * F of Eq. 2 is the parcel force interpolated back to the mesh (Sec. 2.1)
//   * explicit coupling deposits F once per time step; implicit coupling
//     re-deposits it at the head of every gas (SIMPLE) iteration (Sec. 2.2.2)
// The paper leaves drag, interpolation, reflection and the time integrator to
// the MFiX theory guide. The readings used here (trilinear cloud-in-cell
// weights on the node grid; Wen-Yu, Syamlal-O'Brien, Gidaspow or blended
// Gidaspow drag; semi-implicit drag with explicit body and stress forces;
// specular walls at the parcel centre; the gas iteration of implicit coupling
// reduced to the unsteady and drag terms of Eq. 2) are stated at each function.
// Everything is evaluated in the obvious order, one parcel or node at a time,
// in FP64, compiled with FMA contraction disabled so that the binning formula
// is the plain IEEE product.
//
// The step is written once as a template over the scalar type: with S=double
// it is the value oracle; with S=Dual<3> it carries forward-mode tangents with
// respect to (drag multiplier C, diameter scale s_d, inflow velocity u_in),
// which is the oracle gradient of the time-averaged objectives.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

extern "C" {

// Physical and numerical parameters of one bed. Box [0,nx*dx]x[0,ny*dy]x[0,nz*dz].
typedef struct {
  int nx, ny, nz, reserved0;
  double dx, dy, dz;
  double rho_g, mu_g;   // gas density, viscosity
  double g[3];          // gravity
  double gradp[3];      // uniform pressure gradient used when no node field is given
  double rho_p;         // parcel material density
  double Ps, beta, eps_cp, alpha;  // Eq. 5 parameters
  double eps_g_min;     // voidage floor (reading: keeps u_g = U/eps_g and the drag finite)
  double e_wall;        // wall restitution for specular reflection
  double drag_mult;     // C: multiplies the drag coefficient D_p
  double dscale;        // s_d: multiplies every parcel diameter
  double u_in;          // inflow velocity added to the z component of U at every node
  double dt;
  int drag_model;       // 0 Wen-Yu, 1 Syamlal-O'Brien, 2 Gidaspow, 3 Gidaspow blend
  int coupling_iters;   // 0 explicit coupling; K > 0 implicit coupling with K gas iterations
} orc_config;

}  // extern "C"

namespace {

// ---------------------------------------------------------------- scalars --

inline double val(double a) { return a; }

template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0) { for (int i = 0; i < N; ++i) d[i] = 0; }
  Dual(double a) : v(a) { for (int i = 0; i < N; ++i) d[i] = 0; }
};
template <int N> inline double val(const Dual<N>& a) { return a.v; }

template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N>& operator+=(Dual<N>& a, const Dual<N>& b) { a = a + b; return a; }

// a^p for a constant exponent p. At a == 0 the tangent is taken as 0.
inline double powc(double a, double p) { return std::pow(a, p); }
template <int N> inline Dual<N> powc(const Dual<N>& a, double p) {
  Dual<N> r(std::pow(a.v, p));
  double dd = (a.v == 0.0) ? 0.0 : p * std::pow(a.v, p - 1.0);
  for (int i = 0; i < N; ++i) r.d[i] = dd * a.d[i];
  return r; }
// sqrt with the tangent taken as 0 at the origin (zero slip).
inline double sqrtz(double a) { return std::sqrt(a); }
template <int N> inline Dual<N> sqrtz(const Dual<N>& a) {
  Dual<N> r(std::sqrt(a.v));
  double dd = (a.v == 0.0) ? 0.0 : 0.5 / r.v;
  for (int i = 0; i < N; ++i) r.d[i] = dd * a.d[i];
  return r; }
// atan, for the blending function of the Gidaspow blend.
inline double atanv(double a) { return std::atan(a); }
template <int N> inline Dual<N> atanv(const Dual<N>& a) {
  Dual<N> r(std::atan(a.v));
  double dd = 1.0 / (1.0 + a.v * a.v);
  for (int i = 0; i < N; ++i) r.d[i] = dd * a.d[i];
  return r; }
// max/min select one operand by value; the tangent follows the selected operand.
template <class S> inline S maxv(const S& a, const S& b) { return val(a) >= val(b) ? a : b; }
template <class S> inline S minv(const S& a, const S& b) { return val(a) <= val(b) ? a : b; }

template <class S> inline bool finite(const S& a) { return std::isfinite(val(a)); }

// ------------------------------------------------------------------ grid --

struct Grid {
  int n[3];
  double h[3];    // cell size
  double inv[3];  // fl64(1/h): the binning multiplier
  double L[3];    // box length n*h
  long ncell, nnode;
  explicit Grid(const orc_config& c) {
    n[0] = c.nx; n[1] = c.ny; n[2] = c.nz;
    h[0] = c.dx; h[1] = c.dy; h[2] = c.dz;
    for (int a = 0; a < 3; ++a) { inv[a] = 1.0 / h[a]; L[a] = n[a] * h[a]; }
    ncell = (long)n[0] * n[1] * n[2];
    nnode = (long)(n[0] + 1) * (n[1] + 1) * (n[2] + 1);
  }
  long node(int i, int j, int k) const {
    return i + (long)(n[0] + 1) * (j + (long)(n[1] + 1) * k);
  }
  long cell(int i, int j, int k) const { return i + (long)n[0] * (j + (long)n[1] * k); }
  // Control volume of node (i,j,k): the cell volume times 1/2 for each axis on
  // which the node lies on a boundary plane, so the node volumes tile the box.
  double node_volume(int i, int j, int k) const {
    double v = h[0] * h[1] * h[2];
    if (i == 0 || i == n[0]) v *= 0.5;
    if (j == 0 || j == n[1]) v *= 0.5;
    if (k == 0 || k == n[2]) v *= 0.5;
    return v;
  }
};

// Binning along one axis (reading of the paper's cell index tensors, Sec. 2.2.3):
// t = fl64(x * fl64(1/h)); i = clamp(floor(t), 0, n-1); xi = clamp(t - i, 0, 1).
template <class S>
inline void bin_axis(const S& x, double inv, int n, int& i, S& xi) {
  S t = x * inv;
  double f = std::floor(val(t));
  if (!(f >= 0.0)) f = 0.0;               // also catches NaN
  if (f > (double)(n - 1)) f = (double)(n - 1);
  i = (int)f;
  xi = t - f;
  if (val(xi) < 0.0) xi = S(0.0);
  if (val(xi) > 1.0) xi = S(1.0);
}

// Trilinear cloud-in-cell weights of the 8 corners of the parcel's cell and
// their spatial derivatives (reading of the paper's "bilinear" interpolation,
// Sec. 3.1, extended to 3-D). Corner q = a + 2b + 4c sits at node (i+a, j+b, k+c).
template <class S>
struct Stencil {
  int i, j, k;
  long cell;
  long nodes[8];
  S W[8];
  S dW[8][3];
};

template <class S>
inline void stencil(const Grid& G, const S& x, const S& y, const S& z, Stencil<S>& st) {
  S xi, eta, zeta;
  bin_axis(x, G.inv[0], G.n[0], st.i, xi);
  bin_axis(y, G.inv[1], G.n[1], st.j, eta);
  bin_axis(z, G.inv[2], G.n[2], st.k, zeta);
  st.cell = G.cell(st.i, st.j, st.k);
  S wx[2] = {1.0 - xi, xi}, wy[2] = {1.0 - eta, eta}, wz[2] = {1.0 - zeta, zeta};
  const double sx[2] = {-G.inv[0], G.inv[0]}, sy[2] = {-G.inv[1], G.inv[1]},
               sz[2] = {-G.inv[2], G.inv[2]};
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        int q = a + 2 * b + 4 * c;
        st.nodes[q] = G.node(st.i + a, st.j + b, st.k + c);
        st.W[q] = wx[a] * wy[b] * wz[c];
        st.dW[q][0] = sx[a] * (wy[b] * wz[c]);
        st.dW[q][1] = sy[b] * (wx[a] * wz[c]);
        st.dW[q][2] = sz[c] * (wx[a] * wy[b]);
      }
}

// Parcel volume V = w * pi (s_d d)^3 / 6: the statistical weight times the
// volume of one spherical particle (Sec. 2.1).
template <class S>
inline S parcel_volume(double d, double omega, const S& sd) {
  S de = sd * d;
  return omega * (M_PI / 6.0) * (de * de * de);
}

template <class S>
struct Params { S C, sd, uin; };

// Solids volume deposit: Vs_n = sum_p V_p W_pn over each parcel's 8 corners.
template <class S>
void deposit_volume(const Grid& G, const Params<S>& P, long np, const S* x, const S* y,
                    const S* z, const double* d, const double* om, std::vector<S>& Vs) {
  Vs.assign(G.nnode, S(0.0));
  Stencil<S> st;
  for (long p = 0; p < np; ++p) {
    stencil(G, x[p], y[p], z[p], st);
    S V = parcel_volume(d[p], om[p], P.sd);
    for (int q = 0; q < 8; ++q) Vs[st.nodes[q]] += V * st.W[q];
  }
}

// Node fields from the deposited volume: eps_s = Vs / V_node, eps_g = 1 - eps_s,
// interstitial gas velocity u_g = U / max(eps_g, eps_g_min) from the prescribed
// superficial velocity U (plus u_in on z), and the Snider stress of Eq. 5.
template <class S>
void node_fields(const orc_config& c, const Grid& G, const Params<S>& P, const std::vector<S>& Vs,
                 const double* const U[3], std::vector<S>& eps_s, std::vector<S>& ug,
                 std::vector<S>& tau) {
  eps_s.assign(G.nnode, S(0.0));
  ug.assign(3 * G.nnode, S(0.0));
  tau.assign(G.nnode, S(0.0));
  for (int k = 0; k <= G.n[2]; ++k)
    for (int j = 0; j <= G.n[1]; ++j)
      for (int i = 0; i <= G.n[0]; ++i) {
        long n = G.node(i, j, k);
        S es = Vs[n] / G.node_volume(i, j, k);
        S eg = 1.0 - es;
        S egc = maxv(eg, S(c.eps_g_min));
        for (int a = 0; a < 3; ++a) {
          S Ua = S(U[a] ? U[a][n] : 0.0);
          if (a == 2) Ua = Ua + P.uin;
          ug[3 * n + a] = Ua / egc;
        }
        // Eq. 5: tau = p_s eps^beta / max[eps_cp - eps, alpha (1 - eps)]
        S den = maxv(c.eps_cp - es, c.alpha * (1.0 - es));
        tau[n] = c.Ps * powc(es, c.beta) / den;
        eps_s[n] = es;
      }
}

template <class S>
struct Interp { S es, ug[3], gp[3], gt[3]; };

// Grid-to-parcel interpolation with the same weights: eps_s, u_g and grad p
// are weighted sums of node values; grad tau is the exact gradient of the
// trilinear interpolant of the node stresses.
template <class S>
inline void interp(const orc_config& c, const Stencil<S>& st, const std::vector<S>& eps_s,
                   const std::vector<S>& ug, const std::vector<S>& tau,
                   const double* const GP[3], Interp<S>& r) {
  r.es = S(0.0);
  for (int a = 0; a < 3; ++a) { r.ug[a] = S(0.0); r.gt[a] = S(0.0); r.gp[a] = S(0.0); }
  for (int q = 0; q < 8; ++q) {
    long n = st.nodes[q];
    r.es += st.W[q] * eps_s[n];
    for (int a = 0; a < 3; ++a) {
      r.ug[a] += st.W[q] * ug[3 * n + a];
      r.gt[a] += st.dW[q][a] * tau[n];
      if (GP[a]) r.gp[a] += st.W[q] * GP[a][n];
    }
  }
  for (int a = 0; a < 3; ++a)
    if (!GP[a]) r.gp[a] = S(c.gradp[a]);
}

// Wen-Yu drag as an acceleration coefficient: F_P / (eps_P rho_P) = D (u_g - u_P).
//   Re_m = eps_g rho_g d |s| / mu,   Cd = 24/Re_m (1 + 0.15 Re_m^0.687) (Re_m < 1000), else 0.44
//   D = C (3/4) Cd rho_g |s| eps_g^-1.65 / (d rho_p)
// evaluated through Cd|s| so that zero slip stays finite. eps_g is floored at
// eps_g_min (reading).
template <class S>
inline S wen_yu(const orc_config& c, const Params<S>& P, double d, const S& es, const S s[3]) {
  S eg = maxv(1.0 - es, S(c.eps_g_min));
  S de = P.sd * d;
  S smag = sqrtz(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  S Rem = eg * c.rho_g * de * smag / c.mu_g;
  S Cd_s;  // Cd * |s|
  if (val(Rem) < 1000.0)
    Cd_s = 24.0 * c.mu_g / (c.rho_g * de * eg) * (1.0 + 0.15 * powc(Rem, 0.687));
  else
    Cd_s = 0.44 * smag;
  return P.C * 0.75 * Cd_s * c.rho_g * powc(eg, -1.65) / (de * c.rho_p);
}

// Syamlal-O'Brien drag, the closure the paper's runs used (Sec. 2.1), as an acceleration
// coefficient. With the particle Reynolds number Re = rho_g d |s| / mu and the terminal
// velocity ratio of the suspension
//   V_r = (A - 0.06 Re + sqrt((0.06 Re)^2 + 0.12 Re (2B - A) + A^2)) / 2,
//   A = eps_g^4.14,  B = 0.8 eps_g^1.28 (eps_g <= 0.85) or eps_g^2.65 (eps_g > 0.85),
// the drag coefficient is Dallavalle's at the reduced Reynolds number Re / V_r,
//   C_D = (0.63 + 4.8 sqrt(V_r / Re))^2,
// and the exchange coefficient beta = 3/4 C_D eps_s eps_g rho_g |s| / (V_r^2 d) gives
//   D = beta / (eps_s rho_p) = C 3/4 C_D eps_g rho_g |s| / (V_r^2 d rho_p).
// C_D |s| = (0.63 sqrt|s| + 4.8 sqrt(V_r mu / (rho_g d)))^2 keeps zero slip finite.
// V_r is evaluated in the equal form V_r = (A + (A^2 + 2r(2B - A)) / (sqrt(Q) + r)) / 2,
// r = 0.06 Re, Q = r^2 + 2r(2B - A) + A^2 (sqrt(Q) - r rationalised), whose terms are all
// positive (A < 2B for every voidage): the printed form subtracts two numbers of size r and
// loses digits as Re grows. eps_g is floored at eps_g_min as for Wen-Yu (reading).
template <class S>
inline S syamlal_obrien(const orc_config& c, const Params<S>& P, double d, const S& es,
                        const S s[3]) {
  S eg = maxv(1.0 - es, S(c.eps_g_min));
  S de = P.sd * d;
  S smag = sqrtz(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  S Re = c.rho_g * de * smag / c.mu_g;
  S A = powc(eg, 4.14);
  S B = val(eg) <= 0.85 ? 0.8 * powc(eg, 1.28) : powc(eg, 2.65);
  S r = 0.06 * Re;
  S t = A * A + 2.0 * r * (2.0 * B - A);
  S Vr = 0.5 * (A + t / (sqrtz(r * r + t) + r));
  S root = 0.63 * sqrtz(smag) + 4.8 * sqrtz(Vr * c.mu_g / (c.rho_g * de));
  S Cd_s = root * root;  // C_D * |s|
  return P.C * 0.75 * Cd_s * eg * c.rho_g / (Vr * Vr * de * c.rho_p);
}

// Ergun's dense-bed exchange coefficient beta = 150 eps_s^2 mu / (eps_g d^2) +
// 1.75 rho_g eps_s |s| / d as an acceleration coefficient D = beta / (eps_s rho_p), with
// eps_s = 1 - eps_g of the floored voidage (reading).
template <class S>
inline S ergun(const orc_config& c, const Params<S>& P, double d, const S& es, const S s[3]) {
  S eg = maxv(1.0 - es, S(c.eps_g_min));
  S esf = 1.0 - eg;
  S de = P.sd * d;
  S smag = sqrtz(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  return P.C * (150.0 * esf * c.mu_g / (eg * de * de) + 1.75 * c.rho_g * smag / de) / c.rho_p;
}

// Gidaspow drag: Ergun below a voidage of 0.8, Wen-Yu at and above it. The blended form
// (Lu and Gidaspow) weights the two smoothly instead:
//   phi = atan(150 * 1.75 (0.2 - eps_s)) / pi + 1/2,   D = (1 - phi) D_Ergun + phi D_WenYu,
// so dilute suspensions take Wen-Yu and dense beds Ergun.
template <class S>
inline S gidaspow(const orc_config& c, const Params<S>& P, double d, const S& es, const S s[3],
                  bool blend) {
  S eg = maxv(1.0 - es, S(c.eps_g_min));
  if (!blend) return val(eg) < 0.8 ? ergun(c, P, d, es, s) : wen_yu(c, P, d, es, s);
  S phi = atanv(150.0 * 1.75 * (0.2 - (1.0 - eg))) / M_PI + 0.5;
  return (1.0 - phi) * ergun(c, P, d, es, s) + phi * wen_yu(c, P, d, es, s);
}

// The configured drag closure.
template <class S>
inline S drag_coef(const orc_config& c, const Params<S>& P, double d, const S& es, const S s[3]) {
  switch (c.drag_model) {
    case 1: return syamlal_obrien(c, P, d, es, s);
    case 2: return gidaspow(c, P, d, es, s, false);
    case 3: return gidaspow(c, P, d, es, s, true);
    default: return wen_yu(c, P, d, es, s);
  }
}

// Specular reflection at the planes 0 and L, applied to the parcel centre.
// Returns false if the parcel is still outside after one reflection.
template <class S>
inline bool reflect(S& x, S& u, double L, double e) {
  if (val(x) < 0.0) { x = -x; u = -e * u; }
  else if (val(x) > L) { x = 2.0 * L - x; u = -e * u; }
  return val(x) >= 0.0 && val(x) <= L;
}

template <class S>
struct StepOut {
  std::vector<S> Vs, A, B;  // B has 3 entries per node
  S dP, H;
};

// Drag sums of F (Eq. 2) for the parcels at rest in their current state, against the node
// gas velocity ug: per parcel the interpolated fields, the drag coefficient D and
// f = rho_p V D; A = sum_p f W, B = sum_p f u_P W. The parcels do not move.
template <class S>
void drag_sums(const orc_config& c, const Grid& G, const Params<S>& P, long np, const S* x,
               const S* y, const S* z, const S* u, const S* v, const S* w, const double* d,
               const double* om, const std::vector<S>& eps_s, const std::vector<S>& ug,
               const std::vector<S>& tau, const double* const GP[3], std::vector<S>& A,
               std::vector<S>& B) {
  A.assign(G.nnode, S(0.0));
  B.assign(3 * G.nnode, S(0.0));
  Stencil<S> st;
  Interp<S> I;
  for (long p = 0; p < np; ++p) {
    stencil(G, x[p], y[p], z[p], st);
    interp(c, st, eps_s, ug, tau, GP, I);
    S up[3] = {u[p], v[p], w[p]};
    S s[3] = {I.ug[0] - up[0], I.ug[1] - up[1], I.ug[2] - up[2]};
    S f = c.rho_p * parcel_volume(d[p], om[p], P.sd) * drag_coef(c, P, d[p], I.es, s);
    for (int q = 0; q < 8; ++q) {
      long n = st.nodes[q];
      A[n] += f * st.W[q];
      for (int a = 0; a < 3; ++a) B[3 * n + a] += (f * up[a]) * st.W[q];
    }
  }
}

// The gas iteration of implicit coupling (reading of Sec. 2.2.2 with the gas side reduced to
// the unsteady and interphase terms of Eq. 2): per node, backward Euler in the gas velocity
// with the drag force per node volume F = (A u_g - B) / V_n taken implicitly,
//   eps_g rho_g V_n (u_g' - u_g0) / dt = -(A u_g' - B)
//   =>  u_g' = (m u_g0 + B) / (m + A),   m = rho_g eps_g V_n / dt,
// where u_g0 = U / max(eps_g, eps_g_min) is the gas velocity of the time step's start and
// eps_g the floored voidage of the node. Where all four drag sums vanish (no parcel exchanges
// momentum with the node) the update is the identity and u_g0 is kept as it is.
template <class S>
void gas_update(const orc_config& c, const Grid& G, const Params<S>& P, const std::vector<S>& eps_s,
                const double* const U[3], const std::vector<S>& A, const std::vector<S>& B,
                std::vector<S>& ug) {
  for (int k = 0; k <= G.n[2]; ++k)
    for (int j = 0; j <= G.n[1]; ++j)
      for (int i = 0; i <= G.n[0]; ++i) {
        long n = G.node(i, j, k);
        if (val(A[n]) == 0.0 && val(B[3 * n]) == 0.0 && val(B[3 * n + 1]) == 0.0 &&
            val(B[3 * n + 2]) == 0.0)
          continue;
        S egc = maxv(1.0 - eps_s[n], S(c.eps_g_min));
        S m = c.rho_g * egc * G.node_volume(i, j, k) / c.dt;
        for (int a = 0; a < 3; ++a) {
          S Ua = S(U[a] ? U[a][n] : 0.0);
          if (a == 2) Ua = Ua + P.uin;
          S u0 = Ua / egc;
          ug[3 * n + a] = (m * u0 + B[3 * n + a]) / (m + A[n]);
        }
      }
}

// Node fields of a time step's start and, with implicit coupling, the K gas iterations:
// each re-deposits the drag sums against the current gas velocity and updates it.
template <class S>
void coupling(const orc_config& c, const Grid& G, const Params<S>& P, long np, const S* x,
              const S* y, const S* z, const S* u, const S* v, const S* w, const double* d,
              const double* om, const double* const U[3], const double* const GP[3],
              std::vector<S>& Vs, std::vector<S>& eps_s, std::vector<S>& ug, std::vector<S>& tau,
              std::vector<S>& A, std::vector<S>& B) {
  // 1-2: bin and deposit the solids volume at the current positions.
  deposit_volume(G, P, np, x, y, z, d, om, Vs);
  // 3: node fields.
  node_fields(c, G, P, Vs, U, eps_s, ug, tau);
  // implicit coupling: F again at the head of every gas iteration
  for (int m = 0; m < c.coupling_iters; ++m) {
    drag_sums(c, G, P, np, x, y, z, u, v, w, d, om, eps_s, ug, tau, GP, A, B);
    gas_update(c, G, P, eps_s, U, A, B, ug);
  }
}

// The parcel update of parcels [lo, hi) against the node fields of the step's coupling:
// per parcel the interpolation, drag, the drag sums of F (deposited into A, B), the
// objective sums, the push and the walls. Positions/velocities are advanced in place.
// Returns 0, or 4 if a parcel left the box or a value became non-finite.
template <class S>
int push_parcels(const orc_config& c, const Grid& G, const Params<S>& P, long lo, long hi, S* x,
                 S* y, S* z, S* u, S* v, S* w, const double* d, const double* om, int* cell,
                 const double* const GP[3], const std::vector<S>& eps_s, const std::vector<S>& ug,
                 const std::vector<S>& tau, std::vector<S>& A, std::vector<S>& B, S& dPsum,
                 S& Hnum, S& Vsum) {
  int status = 0;
  Stencil<S> st;
  Interp<S> I;
  for (long p = lo; p < hi; ++p) {
    stencil(G, x[p], y[p], z[p], st);
    interp(c, st, eps_s, ug, tau, GP, I);
    S up[3] = {u[p], v[p], w[p]};
    S s[3] = {I.ug[0] - up[0], I.ug[1] - up[1], I.ug[2] - up[2]};
    S D = drag_coef(c, P, d[p], I.es, s);
    S V = parcel_volume(d[p], om[p], P.sd);
    // Drag sums for F of Eq. 2 (pre-push state): A = sum f W, B = sum f u_P W.
    S f = c.rho_p * V * D;
    for (int q = 0; q < 8; ++q) {
      long n = st.nodes[q];
      A[n] += f * st.W[q];
      for (int a = 0; a < 3; ++a) B[3 * n + a] += (f * up[a]) * st.W[q];
    }
    // Objectives: drag momentum delivered to the solids per unit area along z,
    // and twice the volume-weighted mean parcel height.
    dPsum += f * s[2];
    Hnum += V * z[p];
    Vsum += V;
    // Eq. 4 divided by eps_P rho_P; drag implicit, everything else explicit:
    // u* = (u + dt (D u_g + g - grad p / rho_p - grad tau / (eps_s rho_p))) / (1 + dt D)
    // Eq. 3: x* = x + dt u*.
    S pos[3] = {x[p], y[p], z[p]};
    S un[3];
    for (int a = 0; a < 3; ++a) {
      S acc = D * I.ug[a] + c.g[a] - I.gp[a] / c.rho_p;
      if (val(I.es) > 1e-12) acc = acc - I.gt[a] / (I.es * c.rho_p);
      un[a] = (up[a] + c.dt * acc) / (1.0 + c.dt * D);
      pos[a] = pos[a] + c.dt * un[a];
      if (!reflect(pos[a], un[a], G.L[a], c.e_wall)) status = 4;
      if (!finite(pos[a]) || !finite(un[a])) status = 4;
    }
    x[p] = pos[0]; y[p] = pos[1]; z[p] = pos[2];
    u[p] = un[0]; v[p] = un[1]; w[p] = un[2];
    Stencil<S> sn;
    stencil(G, x[p], y[p], z[p], sn);
    if (cell) cell[p] = (int)sn.cell;
  }
  return status;
}

// One coupling step (Sec. 2.2.2): the parcel-to-fluid coupling (once with explicit
// coupling; at the head of every gas iteration with implicit coupling), then the parcel
// update against the last gas velocity, depositing the drag sums F of that update.
// Positions/velocities are advanced in place.
// Returns 0, or 4 if a parcel left the box or a value became non-finite.
template <class S>
int step_once(const orc_config& c, const Grid& G, const Params<S>& P, long np, S* x, S* y, S* z,
              S* u, S* v, S* w, const double* d, const double* om, int* cell,
              const double* const U[3], const double* const GP[3], StepOut<S>& out) {
  std::vector<S> eps_s, ug, tau;
  coupling(c, G, P, np, x, y, z, u, v, w, d, om, U, GP, out.Vs, eps_s, ug, tau, out.A, out.B);
  // 4: per parcel interpolation, drag, drag sums, objectives, push, walls.
  out.A.assign(G.nnode, S(0.0));
  out.B.assign(3 * G.nnode, S(0.0));
  S dPsum(0.0), Hnum(0.0), Vsum(0.0);
  int status = push_parcels(c, G, P, 0, np, x, y, z, u, v, w, d, om, cell, GP, eps_s, ug, tau,
                            out.A, out.B, dPsum, Hnum, Vsum);
  out.dP = dPsum / (G.L[0] * G.L[1]);
  out.H = 2.0 * Hnum / Vsum;
  return status;
}

}  // namespace

extern "C" {

// Cell ids and in-cell coordinates of np parcels (binning formula above).
void orc_bin(const orc_config* c, long np, const double* x, const double* y, const double* z,
             int* cell, double* xi, double* eta, double* zeta) {
  Grid G(*c);
  for (long p = 0; p < np; ++p) {
    int i, j, k;
    double a, b, e;
    bin_axis(x[p], G.inv[0], G.n[0], i, a);
    bin_axis(y[p], G.inv[1], G.n[1], j, b);
    bin_axis(z[p], G.inv[2], G.n[2], k, e);
    if (cell) cell[p] = (int)G.cell(i, j, k);
    if (xi) xi[p] = a;
    if (eta) eta[p] = b;
    if (zeta) zeta[p] = e;
  }
}

// Deposited solids volume per node, Vs[(nx+1)(ny+1)(nz+1)].
void orc_deposit_volume(const orc_config* c, long np, const double* x, const double* y,
                        const double* z, const double* d, const double* om, double* Vs) {
  Grid G(*c);
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  std::vector<double> V;
  deposit_volume(G, P, np, x, y, z, d, om, V);
  std::memcpy(Vs, V.data(), sizeof(double) * G.nnode);
}

// Node fields from a deposited volume: eps_s, u_g (3 arrays) and tau.
// U[a] may be NULL (zero superficial velocity on that axis before u_in).
void orc_node_fields(const orc_config* c, const double* Vs, const double* Ux, const double* Uy,
                     const double* Uz, double* eps_s, double* ugx, double* ugy, double* ugz,
                     double* tau) {
  Grid G(*c);
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  std::vector<double> V(Vs, Vs + G.nnode), es, ug, ta;
  const double* U[3] = {Ux, Uy, Uz};
  node_fields(*c, G, P, V, U, es, ug, ta);
  for (long n = 0; n < G.nnode; ++n) {
    eps_s[n] = es[n]; tau[n] = ta[n];
    ugx[n] = ug[3 * n]; ugy[n] = ug[3 * n + 1]; ugz[n] = ug[3 * n + 2];
  }
}

// Interpolation of node fields to parcels. gp* may be NULL (uniform gradient
// from the config). out has 10 arrays of np: eps_s, ug[3], gradp[3], gradtau[3].
void orc_interp(const orc_config* c, long np, const double* x, const double* y, const double* z,
                const double* eps_s, const double* ugx, const double* ugy, const double* ugz,
                const double* gpx, const double* gpy, const double* gpz, const double* tau,
                double* out) {
  Grid G(*c);
  std::vector<double> es(eps_s, eps_s + G.nnode), ta(tau, tau + G.nnode), ug(3 * G.nnode);
  for (long n = 0; n < G.nnode; ++n) { ug[3 * n] = ugx[n]; ug[3 * n + 1] = ugy[n]; ug[3 * n + 2] = ugz[n]; }
  const double* GP[3] = {gpx, gpy, gpz};
  Stencil<double> st;
  Interp<double> I;
  for (long p = 0; p < np; ++p) {
    stencil(G, x[p], y[p], z[p], st);
    interp(*c, st, es, ug, ta, GP, I);
    out[p] = I.es;
    for (int a = 0; a < 3; ++a) {
      out[(1 + a) * np + p] = I.ug[a];
      out[(4 + a) * np + p] = I.gp[a];
      out[(7 + a) * np + p] = I.gt[a];
    }
  }
}

// Per-parcel drag coefficient D_p (the configured closure) for given interpolated eps_s, u_g.
void orc_drag(const orc_config* c, long np, const double* d, const double* eps_s_p,
              const double* ugx, const double* ugy, const double* ugz, const double* u,
              const double* v, const double* w, double* D) {
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  for (long p = 0; p < np; ++p) {
    double s[3] = {ugx[p] - u[p], ugy[p] - v[p], ugz[p] - w[p]};
    D[p] = drag_coef(*c, P, d[p], eps_s_p[p], s);
  }
}

// The coupling at the start of a time step, without moving the parcels: the deposit, the
// node fields and (with coupling_iters = K > 0) the K gas iterations of implicit coupling.
// Outputs (each may be NULL): Vs, eps_s, the node gas velocity after the iterations
// (ugx, ugy, ugz), tau, and the drag sums of the last gas iteration (A, Bx, By, Bz; zero
// when K = 0).
void orc_couple(const orc_config* c, long np, const double* x, const double* y, const double* z,
                const double* u, const double* v, const double* w, const double* d,
                const double* om, const double* Ux, const double* Uy, const double* Uz,
                const double* gpx, const double* gpy, const double* gpz, double* Vs_out,
                double* es_out, double* ugx, double* ugy, double* ugz, double* tau_out,
                double* A_out, double* Bx, double* By, double* Bz) {
  Grid G(*c);
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  std::vector<double> Vs, eps_s, ug, tau, A(G.nnode, 0.0), B(3 * G.nnode, 0.0);
  const double* U[3] = {Ux, Uy, Uz};
  const double* GP[3] = {gpx, gpy, gpz};
  coupling(*c, G, P, np, x, y, z, u, v, w, d, om, U, GP, Vs, eps_s, ug, tau, A, B);
  for (long n = 0; n < G.nnode; ++n) {
    if (Vs_out) Vs_out[n] = Vs[n];
    if (es_out) es_out[n] = eps_s[n];
    if (ugx) ugx[n] = ug[3 * n];
    if (ugy) ugy[n] = ug[3 * n + 1];
    if (ugz) ugz[n] = ug[3 * n + 2];
    if (tau_out) tau_out[n] = tau[n];
    if (A_out) A_out[n] = A[n];
    if (Bx) Bx[n] = B[3 * n];
    if (By) By[n] = B[3 * n + 1];
    if (Bz) Bz[n] = B[3 * n + 2];
  }
}

// nsteps coupling steps in place. Node arrays (each may be NULL):
//   U[3], gradp[3]   prescribed gas fields at nodes (inputs)
//   Vs               deposited solids volume of the last step (pre-push)
//   A, Bx, By, Bz    drag sums of the last step
//   obj[2*nsteps]    per-step (dP, H)
// Returns 0 or 4 (parcel left the box / non-finite value).
int orc_step(const orc_config* c, long np, double* x, double* y, double* z, double* u, double* v,
             double* w, const double* d, const double* om, int* cell, const double* Ux,
             const double* Uy, const double* Uz, const double* gpx, const double* gpy,
             const double* gpz, int nsteps, double* Vs, double* A, double* Bx, double* By,
             double* Bz, double* obj) {
  Grid G(*c);
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  const double* U[3] = {Ux, Uy, Uz};
  const double* GP[3] = {gpx, gpy, gpz};
  StepOut<double> o;
  int status = 0;
  for (int s = 0; s < nsteps; ++s) {
    int st = step_once(*c, G, P, np, x, y, z, u, v, w, d, om, cell, U, GP, o);
    if (st) status = st;
    if (obj) { obj[2 * s] = o.dP; obj[2 * s + 1] = o.H; }
  }
  if (nsteps > 0) {
    for (long n = 0; n < G.nnode; ++n) {
      if (Vs) Vs[n] = o.Vs[n];
      if (A) A[n] = o.A[n];
      if (Bx) Bx[n] = o.B[3 * n];
      if (By) By[n] = o.B[3 * n + 1];
      if (Bz) Bz[n] = o.B[3 * n + 2];
    }
  }
  return status;
}

// One coupling step of the parcels listed in `sample` (indices into the np parcels), with
// the node fields deposited by all np parcels: the same arithmetic as orc_step for those
// parcels, for checking a large bed on a sample. Outputs per sampled parcel: new x, y, z,
// u, v, w (6 arrays of ns), the new cell id, and its f = rho_p V D. Returns 0 or 4.
int orc_step_sample(const orc_config* c, long np, const double* x, const double* y,
                    const double* z, const double* u, const double* v, const double* w,
                    const double* d, const double* om, const double* Ux, const double* Uy,
                    const double* Uz, long ns, const long* sample, double* out6, int* cell,
                    double* fout) {
  Grid G(*c);
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  std::vector<double> Vs, eps_s, ug, tau, A, B;
  const double* U[3] = {Ux, Uy, Uz};
  const double* GP[3] = {nullptr, nullptr, nullptr};
  coupling(*c, G, P, np, x, y, z, u, v, w, d, om, U, GP, Vs, eps_s, ug, tau, A, B);
  int status = 0;
  Stencil<double> st;
  Interp<double> I;
  for (long t = 0; t < ns; ++t) {
    const long p = sample[t];
    stencil(G, x[p], y[p], z[p], st);
    interp(*c, st, eps_s, ug, tau, GP, I);
    double up[3] = {u[p], v[p], w[p]};
    double s[3] = {I.ug[0] - up[0], I.ug[1] - up[1], I.ug[2] - up[2]};
    double D = drag_coef(*c, P, d[p], I.es, s);
    double V = parcel_volume(d[p], om[p], P.sd);
    fout[t] = c->rho_p * V * D;
    double pos[3] = {x[p], y[p], z[p]};
    for (int a = 0; a < 3; ++a) {
      double acc = D * I.ug[a] + c->g[a] - I.gp[a] / c->rho_p;
      if (I.es > 1e-12) acc = acc - I.gt[a] / (I.es * c->rho_p);
      double un = (up[a] + c->dt * acc) / (1.0 + c->dt * D);
      pos[a] = pos[a] + c->dt * un;
      if (!reflect(pos[a], un, G.L[a], c->e_wall)) status = 4;
      out6[a * ns + t] = pos[a];
      out6[(3 + a) * ns + t] = un;
    }
    Stencil<double> sn;
    stencil(G, pos[0], pos[1], pos[2], sn);
    cell[t] = (int)sn.cell;
  }
  return status;
}

// Forward-mode oracle gradient. Runs nsteps steps carrying tangents with
// respect to theta = (drag_mult, dscale, u_in) and returns
//   out[0..1] = time averages of (dP, H) over the steps,
//   out[2..4] = d<dP>/dtheta,  out[5..7] = d<H>/dtheta.
// The parcel arrays are advanced in place (values only).
int orc_step_tangent(const orc_config* c, long np, double* x, double* y, double* z, double* u,
                     double* v, double* w, const double* d, const double* om, const double* Ux,
                     const double* Uy, const double* Uz, const double* gpx, const double* gpy,
                     const double* gpz, int nsteps, double* out) {
  typedef Dual<3> T;
  Grid G(*c);
  Params<T> P;
  P.C = T(c->drag_mult); P.C.d[0] = 1.0;
  P.sd = T(c->dscale); P.sd.d[1] = 1.0;
  P.uin = T(c->u_in); P.uin.d[2] = 1.0;
  std::vector<T> X(x, x + np), Y(y, y + np), Z(z, z + np), Uu(u, u + np), Vv(v, v + np),
      Ww(w, w + np);
  const double* U[3] = {Ux, Uy, Uz};
  const double* GP[3] = {gpx, gpy, gpz};
  StepOut<T> o;
  T dPm(0.0), Hm(0.0);
  int status = 0;
  for (int s = 0; s < nsteps; ++s) {
    int st = step_once(*c, G, P, np, X.data(), Y.data(), Z.data(), Uu.data(), Vv.data(),
                       Ww.data(), d, om, nullptr, U, GP, o);
    if (st) status = st;
    dPm += o.dP;
    Hm += o.H;
  }
  if (nsteps > 0) { dPm = dPm / (double)nsteps; Hm = Hm / (double)nsteps; }
  out[0] = dPm.v; out[1] = Hm.v;
  for (int i = 0; i < 3; ++i) { out[2 + i] = dPm.d[i]; out[5 + i] = Hm.d[i]; }
  for (long p = 0; p < np; ++p) {
    x[p] = X[p].v; y[p] = Y[p].v; z[p] = Z[p].v; u[p] = Uu[p].v; v[p] = Vv[p].v; w[p] = Ww[p].v;
  }
  return status;
}

}  // extern "C"
