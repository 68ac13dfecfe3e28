// Device compiler of libvqd: native gates and noise processes -> unitaries / superoperators.
//
// Every native operation compiles to exactly ONE operator: noise processes that the paper
// writes as a composition (T1 damping followed by T2 dephasing, Sec. 3.5; the standard error
// deph(p) o depol(q), Eq. (stderr)) are composed here into one superoperator in FP64, so that
// each native op costs one pass over the state.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "vqd_internal.h"

namespace vqd {
namespace {

const double PI = 3.14159265358979323846;
const cd I1(0.0, 1.0);

using Mat = std::vector<cd>;  // row-major square matrix

Mat eye(int d) {
  Mat m(d * d, 0.0);
  for (int i = 0; i < d; i++) m[i * d + i] = 1.0;
  return m;
}
Mat mul(const Mat& a, const Mat& b, int d) {
  Mat c(d * d, 0.0);
  for (int i = 0; i < d; i++)
    for (int l = 0; l < d; l++) {
      cd x = a[i * d + l];
      if (x == 0.0) continue;
      for (int j = 0; j < d; j++) c[i * d + j] += x * b[l * d + j];
    }
  return c;
}
// Kronecker product with `lo` on the low bit(s): (hi (x) lo)[(h1<<b)|l1][(h2<<b)|l2] = hi[h1][h2] lo[l1][l2]
Mat kron(const Mat& hi, int dh, const Mat& lo, int dl) {
  int d = dh * dl;
  Mat m(d * d);
  for (int h1 = 0; h1 < dh; h1++)
    for (int h2 = 0; h2 < dh; h2++)
      for (int l1 = 0; l1 < dl; l1++)
        for (int l2 = 0; l2 < dl; l2++)
          m[(h1 * dl + l1) * d + (h2 * dl + l2)] = hi[h1 * dh + h2] * lo[l1 * dl + l2];
  return m;
}

// Pauli matrices, index 0..3 = I, X, Y, Z
Mat pauli(int s) {
  switch (s) {
    case 0: return {1.0, 0.0, 0.0, 1.0};
    case 1: return {0.0, 1.0, 1.0, 0.0};
    case 2: return {0.0, -I1, I1, 0.0};
    default: return {1.0, 0.0, 0.0, -1.0};
  }
}

// exp(-i a P) for a Pauli product P on two qubits (P^2 = I): cos(a) I - i sin(a) P.
Mat pauli_exp2(int s_lo, int s_hi, double a) {
  Mat P = kron(pauli(s_hi), 2, pauli(s_lo), 2);
  Mat U(16);
  for (int i = 0; i < 16; i++) U[i] = -I1 * std::sin(a) * P[i];
  for (int i = 0; i < 4; i++) U[i * 4 + i] += std::cos(a);
  return U;
}

Mat rot(int axis, double t) {  // exp(-i t sigma_axis / 2)
  Mat P = pauli(axis);
  Mat U(4);
  for (int i = 0; i < 4; i++) U[i] = -I1 * std::sin(t / 2) * P[i];
  U[0] += std::cos(t / 2);
  U[3] += std::cos(t / 2);
  return U;
}

// Raman unitary U(phi, Delta, t) with Rabi frequency Omega, Sec. 6 Eq. (u).
Mat raman(double phi, double om, double de, double t) {
  double w = std::sqrt(om * om + de * de);
  double c = std::cos(w * t / 2), s = std::sin(w * t / 2);
  return {cd(c, -de / w * s), -I1 * (om / w * s) * std::exp(I1 * phi),
          -I1 * (om / w * s) * std::exp(-I1 * phi), cd(c, de / w * s)};
}

// Off-resonant Rabi drive seen by a passive qubit, Sec. 3.3 Eq. (off_resonant), as printed: the detuned
// Rabi rotation exp(-i t (Omega X + Delta Z)/2) followed by the frame phase diag(e^{ih}, e^{-ih}),
// h = Omega_R t / 2, Omega_R = sqrt(Omega^2 + Delta^2).  Omega_R = 0 gives the identity.
Mat off_resonant(double om, double de, double t) {
  const double w = std::hypot(om, de);
  if (w == 0.0) return {1.0, 0.0, 0.0, 1.0};
  const double h = w * t / 2, c = std::cos(h), s = std::sin(h);
  const cd e = std::exp(I1 * h), a(c, -de / w * s), b(0.0, -om / w * s);
  return {a * e, b * e, b / e, std::conj(a) / e};
}

Mat diag4(cd a, cd b, cd c, cd d) {
  Mat m(16, 0.0);
  m[0] = a; m[5] = b; m[10] = c; m[15] = d;
  return m;
}

// ---- superoperators (index s = r | c << k; S = sum conj(K) (x) K with conj on the column part)
Mat sup_kraus(int k, const std::vector<Mat>& ks) {
  int d = 1 << k, D = d * d;
  Mat S(D * D, 0.0);
  for (const Mat& K : ks)
    for (int r1 = 0; r1 < d; r1++)
      for (int c1 = 0; c1 < d; c1++)
        for (int r2 = 0; r2 < d; r2++)
          for (int c2 = 0; c2 < d; c2++)
            S[(r1 | (c1 << k)) * D + (r2 | (c2 << k))] += K[r1 * d + r2] * std::conj(K[c1 * d + c2]);
  return S;
}

// Pauli channel sum_s w_s P_s rho P_s on one (k=1) or two (k=2) qubits, weights indexed by
// s = s_lo + 4 s_hi.  Its superoperator is sum_s w_s conj(P_s) (x) P_s; a Pauli's entries are 0, +-1
// or +-i, so every entry is a signed sum of the weights, formed here without the square roots of a Kraus
// form: the entries that the mathematics makes 1 (for example the populations under a dephasing,
// (1 - p) + p) come out as exactly 1.
Mat sup_pauli(int k, const double* w) {
  const int d = 1 << k, D = d * d, np = k == 1 ? 4 : 16;
  Mat S(D * D, 0.0);
  for (int s = 0; s < np; s++) {
    if (w[s] == 0.0) continue;
    const Mat P = k == 1 ? pauli(s) : kron(pauli(s / 4), 2, pauli(s % 4), 2);
    for (int r1 = 0; r1 < d; r1++)
      for (int c1 = 0; c1 < d; c1++)
        for (int r2 = 0; r2 < d; r2++)
          for (int c2 = 0; c2 < d; c2++) {
            const cd e = P[r1 * d + r2] * std::conj(P[c1 * d + c2]);  // 0, +-1 or +-i, exact
            if (e != 0.0) S[(r1 | (c1 << k)) * D + (r2 | (c2 << k))] += w[s] * e;
          }
  }
  return S;
}

Mat sup_depol1(double p) { double w[4] = {1 - p, p / 3, p / 3, p / 3}; return sup_pauli(1, w); }
Mat sup_deph1(double p) { double w[4] = {1 - p, 0, 0, p}; return sup_pauli(1, w); }
Mat sup_bitflip(double b) { double w[4] = {1 - b, b, 0, 0}; return sup_pauli(1, w); }
Mat sup_depol2(double p) {  // reading of Eq. (depol2): each of the 15 non-identity Pauli pairs with weight p/15
  double w[16];
  for (int s = 0; s < 16; s++) w[s] = s == 0 ? 1 - p : p / 15;
  return sup_pauli(2, w);
}
Mat sup_deph2(double p) {  // Eq. (deph2): Z_i, Z_j, Z_i Z_j with p/3 each
  double w[16] = {0};
  w[0] = 1 - p; w[3] = p / 3; w[12] = p / 3; w[15] = p / 3;
  return sup_pauli(2, w);
}
Mat sup_bitflip2(double b) {  // Eq. (bf2)
  double w[16] = {0};
  w[0] = 1 - b; w[1] = b / 3; w[4] = b / 3; w[5] = b / 3;
  return sup_pauli(2, w);
}
Mat sup_amp(double p) {  // Eq. (damp)
  std::vector<Mat> ks = {{1.0, 0.0, 0.0, std::sqrt(1 - p)}, {0.0, std::sqrt(p), 0.0, 0.0}};
  return sup_kraus(1, ks);
}
Mat sup_gamp(double dt, double t1, double p0) {  // Eq. (gdamp)
  double g = 1 - std::exp(-dt / t1), a = std::sqrt(p0), b = std::sqrt(1 - p0);
  std::vector<Mat> ks = {{a, 0.0, 0.0, a * std::sqrt(1 - g)}, {0.0, a * std::sqrt(g), 0.0, 0.0},
                         {b * std::sqrt(1 - g), 0.0, 0.0, b}, {0.0, 0.0, b * std::sqrt(g), 0.0}};
  return sup_kraus(1, ks);
}

// Superoperator of a product channel: S_lo on the first qubit, S_hi on the second.  The
// 2-qubit superoperator index is s = r0 | r1<<1 | c0<<2 | c1<<3; the 1-qubit ones are r | c<<1.
Mat sup_tensor(const Mat& lo, const Mat& hi) {
  Mat S(256, 0.0);
  for (int a = 0; a < 16; a++)
    for (int b = 0; b < 16; b++) {
      int r0a = a & 1, r1a = (a >> 1) & 1, c0a = (a >> 2) & 1, c1a = (a >> 3) & 1;
      int r0b = b & 1, r1b = (b >> 1) & 1, c0b = (b >> 2) & 1, c1b = (b >> 3) & 1;
      S[a * 16 + b] = lo[(r0a | c0a << 1) * 4 + (r0b | c0b << 1)] * hi[(r1a | c1a << 1) * 4 + (r1b | c1b << 1)];
    }
  return S;
}

// Passive decay pieces, Sec. 3.5.
double t1_amp_p(double dt, double t1) { return 1 - std::exp(-dt / t1); }           // Eq. (ampt1)
double t1_depol_p(double dt, double t1) { return 0.75 * (1 - std::exp(-dt / t1)); } // Eq. (depolt1)
double t2_deph_p(double dt, double t2) { return 0.5 * (1 - std::exp(-dt / t2)); }   // Eq. (depht2)
double t2s_deph_p(double dt, double t2s) {                                            // Eq. (depht2s)
  const double x = dt / t2s;
  return 0.5 * (1 - std::exp(-x * x));
}
double dephasing_time(double t1, double t2, unsigned flags) {
  if (!(flags & VQD_T2_IS_TOTAL)) return t2;
  double inv = 1.0 / t2 - 1.0 / (2.0 * t1);
  if (!(inv > 0)) throw Error(VQD_EINVAL, "T2 > 2 T1 cannot be read as a total coherence time");
  return 1.0 / inv;
}

void require(bool ok, const char* msg) {
  if (!ok) throw Error(VQD_EINVAL, msg);
}

}  // namespace

int native_arity(int code) {
  static const int ar[VQD_OP_COUNT] = {1, 1, 1, 1, 1, 1, 1, 2, 2, 2, 2, 2, 2, 2, 2, 2, 2,
                                       1, 2, 1, 2, 1, 1, 2, 1, 1, 1, 1, 2, 2, 1, 2, 1, 2, 2, 1, 1};
  if (code < 0 || code >= VQD_OP_COUNT) return -1;
  return ar[code];
}

void stderr_params(int nq, double fbar, double x, double* p_deph, double* q_depol) {
  // App. B: F_e = ((d+1) Fbar - 1)/d (Eq. fidelities_relation); with dephasing p = (1-x) eps and
  // depolarising q = x eps, F_e = 1 - p - q + c p q gives c x(1-x) eps^2 - eps + (1 - F_e) = 0,
  // c = 4/3 for one qubit (Eq. fe1) and 16/15 for two.  Smallest non-negative root.
  require(nq == 1 || nq == 2, "stderr: nq must be 1 or 2");
  require(x >= 0 && x <= 1, "stderr: x must be in [0,1]");
  double d = nq == 1 ? 2.0 : 4.0;
  double c = nq == 1 ? 4.0 / 3.0 : 16.0 / 15.0;
  double fe = ((d + 1) * fbar - 1) / d;
  double a = c * x * (1 - x);
  double e1 = 1 - fe, eps;
  if (a == 0.0) {
    eps = e1;
  } else {
    double disc = 1 - 4 * a * e1;
    require(disc >= 0, "stderr: fidelity too low for this error split");
    eps = 2 * e1 / (1 + std::sqrt(disc));  // = (1 - sqrt(disc)) / (2a), stable form
  }
  require(eps >= 0, "stderr: average fidelity above 1");
  *p_deph = (1 - x) * eps;
  *q_depol = x * eps;
}

Op compile_native(const vqd_native_op& o, unsigned flags) {
  int ar = native_arity(o.code);
  require(ar > 0, "unknown native op code");
  require(o.nq == ar, "native op arity does not match its code");
  Op op;
  op.k = ar;
  op.q[0] = o.q[0];
  op.q[1] = ar == 2 ? o.q[1] : 0;
  const double* P = o.par;
  auto U1 = [&](Mat m) { op.unitary = true; op.m = std::move(m); };
  auto S = [&](Mat m) { op.unitary = false; op.m = std::move(m); };
  switch (o.code) {
    case VQD_OP_RX: U1(rot(1, P[0])); break;
    case VQD_OP_RY: U1(rot(2, P[0])); break;
    case VQD_OP_RZ: U1(rot(3, P[0])); break;
    case VQD_OP_SX: U1(rot(1, PI / 2)); break;
    case VQD_OP_H: { double h = 1 / std::sqrt(2.0); U1({h, h, h, -h}); break; }
    case VQD_OP_U: require(std::hypot(P[1], P[2]) > 0, "U: Omega and Delta both zero"); U1(raman(P[0], P[1], P[2], P[3])); break;
    case VQD_OP_R: U1(raman(P[1], 1.0, 0.0, P[0])); break;
    case VQD_OP_CZ: U1(diag4(1, 1, 1, -1)); break;
    case VQD_OP_CPH: U1(diag4(1, 1, 1, std::exp(I1 * P[0]))); break;
    case VQD_OP_CZPHI: U1(diag4(1, std::exp(I1 * P[0]), std::exp(I1 * P[0]), std::exp(I1 * (2 * P[0] - PI)))); break;
    case VQD_OP_ZX: U1(pauli_exp2(3, 1, P[0] / 2)); break;   // Z on the control (first, low bit), X on the target
    case VQD_OP_ZZ: U1(pauli_exp2(3, 3, P[0] / 2)); break;
    case VQD_OP_ZY: U1(pauli_exp2(3, 2, P[0] / 2)); break;  // CRy+-: Z on the control (low bit), Y on the target
    case VQD_OP_XX: U1(pauli_exp2(1, 1, P[0] / 2)); break;
    case VQD_OP_ZZPHASE: U1(pauli_exp2(3, 3, P[0])); break;
    case VQD_OP_ZZ_IDLE: U1(pauli_exp2(3, 3, PI * P[1] * P[0] / 2)); break;  // conditional phase 2 pi xi dt = 4 alpha
    case VQD_OP_CRZ_XTALK: {  // |0><0|_c (x) I + |1><1|_c (x) Rz(alpha); control = low bit
      cd a = std::exp(-I1 * (P[0] / 2)), b = std::exp(I1 * (P[0] / 2));
      // basis index = c | t << 1: |c=0,t=0>, |c=1,t=0>, |c=0,t=1>, |c=1,t=1>
      U1(diag4(1, a, 1, b));
      break;
    }
    case VQD_OP_EXCHANGE: {
      Mat u = mul(mul(pauli_exp2(1, 1, P[0] / 4), pauli_exp2(2, 2, P[0] / 4), 4), pauli_exp2(3, 3, P[0] / 4), 4);
      U1(u);
      break;
    }
    case VQD_OP_OFFRES: U1(off_resonant(P[0], P[1], P[2])); break;
    case VQD_OP_ZZ_STATIC: {  // Sec. 8 static ZZ of a transmon pair; control = first qubit
      const double d1 = P[1] - P[2], d2 = P[1] + P[3];
      require(d1 != 0.0 && d2 != 0.0, "zz_static: Delta_ct - alpha_t or Delta_ct + alpha_c is zero");
      const double beta = P[0] * P[0] * (1.0 / d1 - 1.0 / d2);
      require(std::isfinite(beta), "zz_static: beta is not finite");
      U1(pauli_exp2(3, 3, beta));
      break;
    }
    case VQD_OP_DEPOL1: require(P[0] >= 0 && P[0] <= 0.75 + 1e-12, "depol1: p outside [0,3/4]"); S(sup_depol1(P[0])); break;
    case VQD_OP_DEPOL2: require(P[0] >= 0 && P[0] <= 15.0 / 16 + 1e-12, "depol2: p outside [0,15/16]"); S(sup_depol2(P[0])); break;
    case VQD_OP_DEPH1: require(P[0] >= 0 && P[0] <= 0.5 + 1e-12, "deph1: p outside [0,1/2]"); S(sup_deph1(P[0])); break;
    case VQD_OP_DEPH2: require(P[0] >= 0 && P[0] <= 0.75 + 1e-12, "deph2: p outside [0,3/4]"); S(sup_deph2(P[0])); break;
    case VQD_OP_AMP: require(P[0] >= 0 && P[0] <= 1, "amp: p outside [0,1]"); S(sup_amp(P[0])); break;
    case VQD_OP_BITFLIP: require(P[0] >= 0 && P[0] <= 0.5 + 1e-12, "bitflip: b outside [0,1/2]"); S(sup_bitflip(P[0])); break;
    case VQD_OP_BITFLIP2: require(P[0] >= 0 && P[0] <= 0.75 + 1e-12, "bitflip2: b outside [0,3/4]"); S(sup_bitflip2(P[0])); break;
    case VQD_OP_GAMP:
      require(P[0] >= 0 && P[1] > 0 && P[2] >= 0 && P[2] <= 1, "gamp: need dt >= 0, T1 > 0, p0 in [0,1]");
      S(sup_gamp(P[0], P[1], P[2]));
      break;
    case VQD_OP_IDLE:
    case VQD_OP_IDLE_DEPOL:
    case VQD_OP_AMPDEPH2: {
      require(P[0] >= 0 && P[1] > 0 && P[2] > 0, "idle: need dt >= 0, T1 > 0, T2 > 0");
      double tphi = dephasing_time(P[1], P[2], flags);
      Mat first = o.code == VQD_OP_IDLE_DEPOL ? sup_depol1(t1_depol_p(P[0], P[1])) : sup_amp(t1_amp_p(P[0], P[1]));
      Mat one = mul(sup_deph1(t2_deph_p(P[0], tphi)), first, 4);  // dephasing after the T1 part
      if (o.code == VQD_OP_AMPDEPH2) S(sup_tensor(one, one)); else S(one);
      break;
    }
    case VQD_OP_BITFLIP_ASYM:
      require(P[0] >= 0 && P[0] <= 1 && P[1] >= 0 && P[1] <= 1, "bitflip_asym: p10, p01 outside [0,1]");
      S(sup_kraus(1, {{std::sqrt(1 - P[1]), 0.0, 0.0, std::sqrt(1 - P[0])}, {0.0, std::sqrt(P[0]), 0.0, 0.0},
                      {0.0, 0.0, std::sqrt(P[1]), 0.0}}));
      break;
    case VQD_OP_IDLE_T2S:
      require(P[0] >= 0 && P[1] > 0 && P[2] > 0, "idle_t2s: need dt >= 0, T1 > 0, T2* > 0");
      S(mul(sup_deph1(t2s_deph_p(P[0], P[2])), sup_depol1(t1_depol_p(P[0], P[1])), 4));  // dephasing after T1
      break;
    case VQD_OP_STDERR1:
    case VQD_OP_STDERR2: {
      double p, q;
      stderr_params(ar, P[0], P[1], &p, &q);
      Mat dep = ar == 1 ? sup_depol1(q) : sup_depol2(q);
      Mat dph = ar == 1 ? sup_deph1(p) : sup_deph2(p);
      S(mul(dph, dep, ar == 1 ? 4 : 16));  // Eq. (stderr): deph(p) o depol(q)
      break;
    }
    case VQD_OP_LEAK_INIT: {
      require(P[0] >= 0 && P[0] <= 1, "leak_init: gamma outside [0,1]");
      S(sup_kraus(1, {{std::sqrt(1 - P[0]), 0.0, 0.0, 1.0}}));
      break;
    }
    case VQD_OP_LEAK_CZ: {
      require(P[0] >= 0 && P[0] <= 1 && P[1] >= 0 && P[1] <= 1, "leak_cz: alpha, beta outside [0,1]");
      S(sup_kraus(2, {diag4(1.0, std::sqrt(1 - P[0]), std::sqrt(1 - P[0]), std::sqrt(1 - P[1]))}));
      break;
    }
    default: throw Error(VQD_EINVAL, "unknown native op code");
  }
  return op;
}

std::vector<cd> superop_from_kraus(int k, int nK, const cd* K) {
  int d = 1 << k;
  std::vector<Mat> ks;
  for (int j = 0; j < nK; j++) ks.emplace_back(K + j * d * d, K + (j + 1) * d * d);
  return sup_kraus(k, ks);
}

// A diagonal unitary has |U_rr| = 1, so its superoperator's factors U_rr conj(U_cc) are exactly 1
// whenever U_rr and U_cc are the same number (always for r = c; for r != c in phases such as ZZ or CPh);
// they are set to 1 rather than to the rounded product, which lets the elementwise passes leave those
// members untouched.
bool is_diagonal_matrix(int d, const cd* M) {
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++)
      if (i != j && M[i * d + j] != 0.0) return false;
  return true;
}

std::vector<cd> superop_from_unitary(int k, const cd* U) {
  int d = 1 << k;
  std::vector<cd> S = sup_kraus(k, {Mat(U, U + d * d)});
  if (is_diagonal_matrix(d, U))
    for (int r = 0; r < d; r++)
      for (int c = 0; c < d; c++) {
        const int s = r | (c << k);
        S[(size_t)s * d * d + s] = diag_unitary_factor(U[r * d + r], U[c * d + c]);
      }
  return S;
}

void check_unitary(int k, const cd* U) {
  int d = 1 << k;
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      cd s = 0;
      for (int l = 0; l < d; l++) s += std::conj(U[l * d + i]) * U[l * d + j];
      if (std::abs(s - (i == j ? 1.0 : 0.0)) > 1e-10) throw Error(VQD_ENOTCP, "matrix is not unitary (tol 1e-10)");
    }
}

// Largest eigenvalue of a Hermitian d x d matrix (d <= 4) by cyclic Jacobi on its real
// symmetric 2d x 2d embedding [[Re, -Im], [Im, Re]] (same spectrum, each eigenvalue twice).
static double max_eig_hermitian(int d, const cd* H) {
  int m = 2 * d;
  double A[8][8];
  for (int i = 0; i < d; i++)
    for (int j = 0; j < d; j++) {
      cd h = 0.5 * (H[i * d + j] + std::conj(H[j * d + i]));
      A[i][j] = h.real(); A[i + d][j + d] = h.real();
      A[i][j + d] = -h.imag(); A[i + d][j] = h.imag();
    }
  for (int sweep = 0; sweep < 60; sweep++) {
    double off = 0;
    for (int i = 0; i < m; i++)
      for (int j = i + 1; j < m; j++) off += A[i][j] * A[i][j];
    if (off < 1e-30) break;
    for (int p = 0; p < m; p++)
      for (int q = p + 1; q < m; q++) {
        if (std::fabs(A[p][q]) < 1e-300) continue;
        double th = (A[q][q] - A[p][p]) / (2 * A[p][q]);
        double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1));
        double c = 1 / std::sqrt(t * t + 1), s = t * c;
        for (int r = 0; r < m; r++) {  // columns p, q
          double arp = A[r][p], arq = A[r][q];
          A[r][p] = c * arp - s * arq;
          A[r][q] = s * arp + c * arq;
        }
        for (int r = 0; r < m; r++) {  // rows p, q
          double apr = A[p][r], aqr = A[q][r];
          A[p][r] = c * apr - s * aqr;
          A[q][r] = s * apr + c * aqr;
        }
      }
  }
  double mx = A[0][0];
  for (int i = 1; i < m; i++) mx = std::max(mx, A[i][i]);
  return mx;
}

void check_cptn(int k, int nK, const cd* K) {
  int d = 1 << k;
  std::vector<cd> M(d * d, 0.0);  // sum K^dagger K - I
  for (int j = 0; j < nK; j++)
    for (int a = 0; a < d; a++)
      for (int b = 0; b < d; b++)
        for (int l = 0; l < d; l++) M[a * d + b] += std::conj(K[j * d * d + l * d + a]) * K[j * d * d + l * d + b];
  for (int a = 0; a < d; a++) M[a * d + a] -= 1.0;
  if (max_eig_hermitian(d, M.data()) > 1e-10)
    throw Error(VQD_ENOTCP, "Kraus set is not trace non-increasing: sum K^dagger K exceeds I by more than 1e-10");
}

// Choose the plain-path kernel for one operator.
Pass classify(const Op& op) {
  Pass p;
  p.k = op.k;
  p.q[0] = op.q[0];
  p.q[1] = op.q[1];
  p.weight = op.weight;
  int d = 1 << op.k, D = d * d;
  if (op.unitary) {
    bool diag = true;
    for (int i = 0; i < d; i++)
      for (int j = 0; j < d; j++)
        if (i != j && op.m[i * d + j] != 0.0) diag = false;
    if (diag) {  // factor for amplitude (r, c): U[r][r] conj(U[c][c]), exactly 1 when the entries are equal
      p.kind = KK_ELEM;
      p.coef.resize(D);
      for (int r = 0; r < d; r++)
        for (int c = 0; c < d; c++) p.coef[r | (c << op.k)] = diag_unitary_factor(op.m[r * d + r], op.m[c * d + c]);
      return p;
    }
    if (op.k == 1) {
      p.kind = KK_SUP1;
      p.coef = superop_from_unitary(1, op.m.data());
      return p;
    }
    p.kind = KK_UNI2;
    p.coef = op.m;
    return p;
  }
  bool diag = true;
  for (int i = 0; i < D; i++)
    for (int j = 0; j < D; j++)
      if (i != j && op.m[i * D + j] != 0.0) diag = false;
  if (diag) {
    p.kind = KK_ELEM;
    p.coef.resize(D);
    for (int i = 0; i < D; i++) p.coef[i] = op.m[i * D + i];
    return p;
  }
  p.kind = op.k == 1 ? KK_SUP1 : KK_SUP2;
  p.coef = op.m;
  return p;
}

// ================================================================== Kraus forms (trajectory path)
namespace {

Mat scaled(const Mat& m, double a) {
  Mat r(m);
  for (cd& x : r) x *= a;
  return r;
}
std::vector<Mat> kraus_pauli1(const double* w) {  // order I, X, Y, Z; zero weights dropped
  std::vector<Mat> ks;
  for (int s = 0; s < 4; s++)
    if (w[s] > 0) ks.push_back(scaled(pauli(s), std::sqrt(w[s])));
  return ks;
}
Mat two(const Mat& lo, const Mat& hi) { return kron(hi, 2, lo, 2); }
std::vector<Mat> kraus_depol2(double p) {  // low qubit's Pauli outer, high qubit's inner
  std::vector<Mat> ks;
  for (int a = 0; a < 4; a++)
    for (int b = 0; b < 4; b++) {
      double w = (a == 0 && b == 0) ? 1 - p : p / 15;
      if (w > 0) ks.push_back(scaled(two(pauli(a), pauli(b)), std::sqrt(w)));
    }
  return ks;
}
std::vector<Mat> kraus_three2(double p, int s) {  // (1-p) I + p/3 (S (x) I, I (x) S, S (x) S), S = pauli(s)
  std::vector<Mat> ks = {scaled(eye(4), std::sqrt(1 - p))};
  if (p > 0) {
    ks.push_back(scaled(two(pauli(s), pauli(0)), std::sqrt(p / 3)));
    ks.push_back(scaled(two(pauli(0), pauli(s)), std::sqrt(p / 3)));
    ks.push_back(scaled(two(pauli(s), pauli(s)), std::sqrt(p / 3)));
  }
  return ks;
}
std::vector<Mat> kraus_amp(double p) { return {{1.0, 0.0, 0.0, std::sqrt(1 - p)}, {0.0, std::sqrt(p), 0.0, 0.0}}; }
std::vector<Mat> kraus_then(const std::vector<Mat>& first, const std::vector<Mat>& second, int d) {
  std::vector<Mat> ks;
  for (const Mat& A : first)
    for (const Mat& B : second) ks.push_back(mul(B, A, d));
  return ks;
}

}  // namespace

KrausForm compile_kraus_form(const vqd_native_op& o, unsigned flags) {
  Op op = compile_native(o, flags);  // validates the op; gives U for unitaries
  KrausForm f;
  f.k = op.k;
  f.q[0] = op.q[0];
  f.q[1] = op.q[1];
  if (op.unitary) {
    f.unitary = true;
    f.K = {op.m};
    return f;
  }
  f.unitary = false;
  const double* P = o.par;
  switch (o.code) {
    case VQD_OP_DEPOL1: { double w[4] = {1 - P[0], P[0] / 3, P[0] / 3, P[0] / 3}; f.K = kraus_pauli1(w); break; }
    case VQD_OP_DEPH1: { double w[4] = {1 - P[0], 0, 0, P[0]}; f.K = kraus_pauli1(w); break; }
    case VQD_OP_BITFLIP: { double w[4] = {1 - P[0], P[0], 0, 0}; f.K = kraus_pauli1(w); break; }
    case VQD_OP_DEPOL2: f.K = kraus_depol2(P[0]); break;
    case VQD_OP_DEPH2: f.K = kraus_three2(P[0], 3); break;
    case VQD_OP_BITFLIP2: f.K = kraus_three2(P[0], 1); break;
    case VQD_OP_AMP: f.K = kraus_amp(P[0]); break;
    case VQD_OP_GAMP: {
      double g = 1 - std::exp(-P[0] / P[1]), a = std::sqrt(P[2]), b = std::sqrt(1 - P[2]);
      f.K = {{a, 0.0, 0.0, a * std::sqrt(1 - g)}, {0.0, a * std::sqrt(g), 0.0, 0.0},
             {b * std::sqrt(1 - g), 0.0, 0.0, b}, {0.0, 0.0, b * std::sqrt(g), 0.0}};
      break;
    }
    case VQD_OP_IDLE:
    case VQD_OP_IDLE_DEPOL:
    case VQD_OP_AMPDEPH2: {
      double tphi = dephasing_time(P[1], P[2], flags);
      double pd = t2_deph_p(P[0], tphi);
      double wd[4] = {1 - pd, 0, 0, pd};
      std::vector<Mat> first;
      if (o.code == VQD_OP_IDLE_DEPOL) {
        double q = t1_depol_p(P[0], P[1]);
        double w[4] = {1 - q, q / 3, q / 3, q / 3};
        first = kraus_pauli1(w);
      } else {
        first = kraus_amp(t1_amp_p(P[0], P[1]));
      }
      std::vector<Mat> one = kraus_then(first, kraus_pauli1(wd), 2);
      if (o.code == VQD_OP_AMPDEPH2) {
        for (const Mat& A : one)
          for (const Mat& B : one) f.K.push_back(two(A, B));
      } else {
        f.K = one;
      }
      break;
    }
    case VQD_OP_BITFLIP_ASYM:
      f.K = {{std::sqrt(1 - P[1]), 0.0, 0.0, std::sqrt(1 - P[0])}, {0.0, std::sqrt(P[0]), 0.0, 0.0},
             {0.0, 0.0, std::sqrt(P[1]), 0.0}};
      break;
    case VQD_OP_IDLE_T2S: {
      const double q = t1_depol_p(P[0], P[1]), pd = t2s_deph_p(P[0], P[2]);
      double wq[4] = {1 - q, q / 3, q / 3, q / 3}, wd[4] = {1 - pd, 0, 0, pd};
      f.K = kraus_then(kraus_pauli1(wq), kraus_pauli1(wd), 2);
      break;
    }
    case VQD_OP_STDERR1:
    case VQD_OP_STDERR2: {
      double p, q;
      stderr_params(op.k, P[0], P[1], &p, &q);
      if (op.k == 1) {
        double wq[4] = {1 - q, q / 3, q / 3, q / 3}, wp[4] = {1 - p, 0, 0, p};
        f.K = kraus_then(kraus_pauli1(wq), kraus_pauli1(wp), 2);
      } else {
        f.K = kraus_then(kraus_depol2(q), kraus_three2(p, 3), 4);
      }
      break;
    }
    case VQD_OP_LEAK_INIT: f.K = {{std::sqrt(1 - P[0]), 0.0, 0.0, 1.0}}; break;
    case VQD_OP_LEAK_CZ: f.K = {diag4(1.0, std::sqrt(1 - P[0]), std::sqrt(1 - P[0]), std::sqrt(1 - P[1]))}; break;
    default: throw Error(VQD_EINVAL, "no Kraus form for this op");
  }
  // state-independent branch probabilities: K_k^dagger K_k = w_k I for every k
  const int d = 1 << op.k;
  f.mixture = true;
  for (const Mat& K : f.K) {
    double w = 0;
    for (int i = 0; i < d * d; i++) w += std::norm(K[i]);
    w /= d;
    for (int a = 0; a < d && f.mixture; a++)
      for (int b = 0; b < d; b++) {
        cd s = 0;
        for (int l = 0; l < d; l++) s += std::conj(K[l * d + a]) * K[l * d + b];
        if (std::abs(s - (a == b ? w : 0.0)) > 1e-12) {
          f.mixture = false;
          break;
        }
      }
    f.w.push_back(w);
  }
  if (!f.mixture) f.w.clear();
  return f;
}

}  // namespace vqd
