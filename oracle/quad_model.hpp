// TEST INFRASTRUCTURE ONLY: the slow, plain FP64 definition of one step of
// the batched quadrotor model that the CUDA library is checked against.  It is
// written agent by agent, in the order of the equations, with no blocking or
// fusion.  Only tests, the smoke check and the CPU-baseline leg of the bench
// use it.  It shares no code with the CUDA library.
//
// Passages followed (arXiv 2308.12698, Sec. III-B "Quadrotor Dynamics &
// Control"):
//   Eq. (qd1)  p' = v
//   Eq. (qd2)  v' = R(q) f_u / m + g,  f_u = [0, 0, f_c],  g = [0, 0, -g]
//   Eq. (qd3)  q' = 1/2 q o [0, omega]        (Hamilton product)
//   Eq. (qd4)  omega' = I^-1 (-omega x (I omega) + tau_u),  I = diag
//   Eq. (2)    f_i = k_t Omega_i^2,  tau_i = k_q Omega_i^2
//   Eq. (3)    [f_c, tau_x, tau_y, tau_z] = G [f_1..f_4]   (G as printed)
//   RK4 discretisation (end of Sec. III-B); body-rate inner loop (same place).
// The paper leaves the following to the workload definition; the readings
// taken here are:
//   * rotor speeds are states with a first-order lag Omega' = (Omega_cmd - Omega)/tau_m;
//   * linear drag -c_d v is added to m v';
//   * Omega is in rad/s (the paper's "RPM" would make hover 606 RPM);
//   * L is the centre-to-rotor distance and alpha the arm angle from body x;
//   * the controller is a cascade evaluated once per step and held over the
//     four RK4 stages: position PD with per-axis acceleration clamp and
//     gravity feed-forward -> desired attitude from the thrust direction and
//     heading -> attitude P on the error quaternion -> body-rate P scaled by
//     the maximum torque per axis -> inverse allocation G^-1 -> per-rotor
//     clamp of Omega^2 to [0, Omega_max^2] -> square root;
//   * no quaternion renormalisation;
//   * PID variant of the body-rate loop (mode CLOSED_LOOP_PID; the paper names
//     a "PID body rate controller" and gives no gains): per axis
//     tau_i = taumax_i (krate_i e_i + kI_i xi_i - kD_i omega'_i) with the rate
//     error e = omega_des - omega, the integral xi of e as three extra states
//     (20 in all), advanced once per step by xi <- clamp(xi + h e, +-xi_max)
//     and held over the RK4 stages like the command, and the derivative taken
//     on the measurement: omega' of Eq. (qd4) at the step start.  kI = kD = 0
//     gives the P loop exactly.
#pragma once
#include <cmath>
#include "scalar_types.hpp"

namespace orc {

constexpr int NX = 17;      // p(3) v(3) q(4: w x y z) omega(3) Omega(4)
constexpr int NXP = 20;     // PID mode: the 17 plus the rate-error integral xi(3)
constexpr int NPARAM = 43;  // packed parameter group (see unpack_group)
constexpr int NTHETA = 16;  // kp(3) kd(3) katt(3) krate(3) m Jxx Jyy Jzz
enum { OPEN_LOOP = 0, CLOSED_LOOP = 1, CLOSED_LOOP_PID = 2 };

inline int state_dim(int mode) { return mode == CLOSED_LOOP_PID ? NXP : NX; }

template <class T>
struct Group {
  T m, J[3];              // mass, principal inertias Ixx Iyy Izz
  T L, alpha;             // arm length, arm angle (geometry of G in Eq. 3)
  T kt, kq;               // Eq. 2 coefficients
  T tau_m, c_d, omega_max, g;
  T kp[3], kd[3], katt[3], krate[3];
  T a_max;
  T kI[3], kD[3], xi_max[3];  // PID mode only
  int type = 0;                // agent type: 0 quadrotor, 1 car, 2 fixed-wing (vehicles.hpp)
  double veh[8] = {};          // parameters of the car or fixed-wing model
};

// Packed order: m Jxx Jyy Jzz L alpha kt kq tau_m c_d omega_max g kp[3] kd[3]
// katt[3] krate[3] a_max kI[3] kD[3] xi_max[3] type veh[8].
inline Group<double> unpack_group(const double* p) {
  Group<double> G;
  G.m = p[0];
  for (int i = 0; i < 3; ++i) G.J[i] = p[1 + i];
  G.L = p[4]; G.alpha = p[5]; G.kt = p[6]; G.kq = p[7];
  G.tau_m = p[8]; G.c_d = p[9]; G.omega_max = p[10]; G.g = p[11];
  for (int i = 0; i < 3; ++i) {
    G.kp[i] = p[12 + i]; G.kd[i] = p[15 + i]; G.katt[i] = p[18 + i]; G.krate[i] = p[21 + i];
  }
  G.a_max = p[24];
  for (int i = 0; i < 3; ++i) {
    G.kI[i] = p[25 + i]; G.kD[i] = p[28 + i]; G.xi_max[i] = p[31 + i];
  }
  G.type = (int)p[34];
  for (int i = 0; i < 8; ++i) G.veh[i] = p[35 + i];
  return G;
}

template <class T, class S>
Group<T> cast_group(const Group<S>& s) {
  Group<T> G;
  G.m = T(val(s.m));
  for (int i = 0; i < 3; ++i) G.J[i] = T(val(s.J[i]));
  G.L = T(val(s.L)); G.alpha = T(val(s.alpha)); G.kt = T(val(s.kt)); G.kq = T(val(s.kq));
  G.tau_m = T(val(s.tau_m)); G.c_d = T(val(s.c_d)); G.omega_max = T(val(s.omega_max)); G.g = T(val(s.g));
  for (int i = 0; i < 3; ++i) {
    G.kp[i] = T(val(s.kp[i])); G.kd[i] = T(val(s.kd[i]));
    G.katt[i] = T(val(s.katt[i])); G.krate[i] = T(val(s.krate[i]));
  }
  G.a_max = T(val(s.a_max));
  for (int i = 0; i < 3; ++i) {
    G.kI[i] = T(val(s.kI[i])); G.kD[i] = T(val(s.kD[i])); G.xi_max[i] = T(val(s.xi_max[i]));
  }
  G.type = s.type;
  for (int i = 0; i < 8; ++i) G.veh[i] = s.veh[i];
  return G;
}

// Per-group constants that do not depend on the differentiated parameters:
// the allocation matrix of Eq. 3 as printed, its inverse, and the largest
// body torque each axis can produce inside the rotor clamp.
struct Fixed {
  double G[4][4];
  double Ginv[4][4];
  double taumax[3];
};

// Gauss-Jordan inverse with partial pivoting (a plain library-style routine).
inline bool invert4(const double A[4][4], double Ainv[4][4]) {
  double M[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 8; ++c) M[r][c] = c < 4 ? A[r][c] : (c - 4 == r ? 1.0 : 0.0);
  for (int col = 0; col < 4; ++col) {
    int piv = col;
    for (int r = col + 1; r < 4; ++r)
      if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return false;
    if (piv != col)
      for (int c = 0; c < 8; ++c) std::swap(M[piv][c], M[col][c]);
    const double d = M[col][col];
    for (int c = 0; c < 8; ++c) M[col][c] /= d;
    for (int r = 0; r < 4; ++r) {
      if (r == col) continue;
      const double f = M[r][col];
      for (int c = 0; c < 8; ++c) M[r][c] -= f * M[col][c];
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) Ainv[r][c] = M[r][c + 4];
  return true;
}

inline Fixed make_fixed(const Group<double>& P) {
  Fixed F;
  const double s = P.L * std::sin(P.alpha), c = P.L * std::cos(P.alpha), r = P.kq / P.kt;
  const double G[4][4] = {{1, 1, 1, 1}, {s, -s, -s, s}, {-c, -c, c, c}, {r, -r, r, -r}};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) F.G[i][j] = G[i][j];
  invert4(F.G, F.Ginv);
  // Largest |tau| per axis with every f_i in [0, kt Omega_max^2]: the rotors
  // on the positive side of a row at full thrust, the others at zero.
  const double fmax = P.kt * P.omega_max * P.omega_max;
  for (int a = 0; a < 3; ++a) {
    double t = 0.0;
    for (int j = 0; j < 4; ++j)
      if (F.G[a + 1][j] > 0) t += F.G[a + 1][j] * fmax;
    F.taumax[a] = t;
  }
  return F;
}

// ---------------------------------------------------------------- helpers --
template <class T>
void hamilton(const T a[4], const T b[4], T o[4]) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

template <class T>
void cross(const T a[3], const T b[3], T o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Rotation matrix of a unit quaternion (body -> inertial), standard form.
template <class T>
void quat_to_R(const T q[4], T R[3][3]) {
  const T w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = T(1.0) - T(2.0) * (y * y + z * z);
  R[0][1] = T(2.0) * (x * y - w * z);
  R[0][2] = T(2.0) * (x * z + w * y);
  R[1][0] = T(2.0) * (x * y + w * z);
  R[1][1] = T(1.0) - T(2.0) * (x * x + z * z);
  R[1][2] = T(2.0) * (y * z - w * x);
  R[2][0] = T(2.0) * (x * z - w * y);
  R[2][1] = T(2.0) * (y * z + w * x);
  R[2][2] = T(1.0) - T(2.0) * (x * x + y * y);
}

// Third column of R(q): the body z axis in the inertial frame.
template <class T>
void body_z(const T q[4], T b3[3]) {
  const T w = q[0], x = q[1], y = q[2], z = q[3];
  b3[0] = T(2.0) * (x * z + w * y);
  b3[1] = T(2.0) * (y * z - w * x);
  b3[2] = T(1.0) - T(2.0) * (x * x + y * y);
}

template <class T>
T clampv(T x, double lo, double hi) {
  const double v = val(x);
  if (v < lo) return T(lo);
  if (v > hi) return T(hi);
  return x;
}

// Unit quaternion of a rotation matrix (Shepperd's method): the scalar branch
// when the trace is positive, otherwise the branch of the largest diagonal
// entry (ties to the lowest index x, y, z).
template <class T>
void shepperd(const T R[3][3], T q[4]) {
  const double tr = val(R[0][0]) + val(R[1][1]) + val(R[2][2]);
  if (tr > 0.0) {
    const T r = sqrt(T(1.0) + R[0][0] + R[1][1] + R[2][2]);
    const T k = T(0.5) / r;
    q[0] = T(0.5) * r;
    q[1] = (R[2][1] - R[1][2]) * k;
    q[2] = (R[0][2] - R[2][0]) * k;
    q[3] = (R[1][0] - R[0][1]) * k;
    return;
  }
  int i = 0;
  if (val(R[1][1]) > val(R[i][i])) i = 1;
  if (val(R[2][2]) > val(R[i][i])) i = 2;
  if (i == 0) {
    const T r = sqrt(T(1.0) + R[0][0] - R[1][1] - R[2][2]);
    const T k = T(0.5) / r;
    q[1] = T(0.5) * r;
    q[0] = (R[2][1] - R[1][2]) * k;
    q[2] = (R[0][1] + R[1][0]) * k;
    q[3] = (R[0][2] + R[2][0]) * k;
  } else if (i == 1) {
    const T r = sqrt(T(1.0) - R[0][0] + R[1][1] - R[2][2]);
    const T k = T(0.5) / r;
    q[2] = T(0.5) * r;
    q[0] = (R[0][2] - R[2][0]) * k;
    q[1] = (R[0][1] + R[1][0]) * k;
    q[3] = (R[1][2] + R[2][1]) * k;
  } else {
    const T r = sqrt(T(1.0) - R[0][0] - R[1][1] + R[2][2]);
    const T k = T(0.5) / r;
    q[3] = T(0.5) * r;
    q[0] = (R[1][0] - R[0][1]) * k;
    q[1] = (R[0][2] + R[2][0]) * k;
    q[2] = (R[1][2] + R[2][1]) * k;
  }
}

// -------------------------------------------------------------- the model --

// Rotor thrusts (Eq. 2) and their resultant through G (Eq. 3), each printed
// row of G written out: u = [f_c, tau_x, tau_y, tau_z].
template <class T>
void rotor_wrench(const Group<T>& P, const Fixed& F, const T Om[4], T u[4]) {
  T f[4];
  for (int i = 0; i < 4; ++i) f[i] = P.kt * (Om[i] * Om[i]);
  const double s = F.G[1][0], c = F.G[2][2], r = F.G[3][0];
  u[0] = f[0] + f[1] + f[2] + f[3];
  u[1] = T(s) * (f[0] - f[1] - f[2] + f[3]);
  u[2] = T(c) * (-f[0] - f[1] + f[2] + f[3]);
  u[3] = T(r) * (f[0] - f[1] + f[2] - f[3]);
}

// Time derivative of the 17-state for held rotor commands w (rad/s).
template <class T>
void derivative(const Group<T>& P, const Fixed& F, const T x[NX], const T w[4], T dx[NX]) {
  const T* p = x;
  const T* v = x + 3;
  const T* q = x + 6;
  const T* om = x + 10;
  const T* Om = x + 13;
  (void)p;
  T u[4];
  rotor_wrench(P, F, Om, u);
  // Eq. (qd1)
  for (int i = 0; i < 3; ++i) dx[i] = v[i];
  // Eq. (qd2) with linear drag: v' = R(q) [0,0,f_c]/m - (c_d/m) v + [0,0,-g]
  T b3[3];
  body_z(q, b3);
  const T acc = u[0] / P.m;
  const T drag = P.c_d / P.m;
  for (int i = 0; i < 3; ++i) dx[3 + i] = b3[i] * acc - drag * v[i];
  dx[5] = dx[5] - P.g;
  // Eq. (qd3): q' = 1/2 q o [0, omega]
  const T wq[4] = {T(0.0), om[0], om[1], om[2]};
  T qd[4];
  hamilton(q, wq, qd);
  for (int i = 0; i < 4; ++i) dx[6 + i] = T(0.5) * qd[i];
  // Eq. (qd4): omega' = I^-1 (-omega x (I omega) + tau)
  const T Iw[3] = {P.J[0] * om[0], P.J[1] * om[1], P.J[2] * om[2]};
  T gyro[3];
  cross(om, Iw, gyro);
  for (int i = 0; i < 3; ++i) dx[10 + i] = (u[1 + i] - gyro[i]) / P.J[i];
  // first-order rotor lag
  for (int i = 0; i < 4; ++i) dx[13 + i] = (w[i] - Om[i]) / P.tau_m;
}

// Cascaded controller: state and waypoint command -> rotor speed commands.
// Optional diagnostics (no effect on the result): the unclamped acceleration
// demand ar[3] and the unclamped rotor demand S[4] = Omega_cmd^2 before the
// clamp to [0, omega_max^2].  PID rate loop when xi (the rate-error integral)
// and wdot (omega' at this state) are given; e_out receives the rate error.
template <class T>
void controller(const Group<T>& P, const Fixed& F, const T x[NX], const double cmd[4], T w[4],
                double* ar_out = nullptr, double* S_out = nullptr, const T* xi = nullptr,
                const T* wdot = nullptr, T* e_out = nullptr) {
  const T* p = x;
  const T* v = x + 3;
  const T* q = x + 6;
  const T* om = x + 10;
  // position PD with per-axis acceleration clamp, gravity feed-forward
  T Fd[3];
  for (int i = 0; i < 3; ++i) {
    const T e = T(cmd[i]) - p[i];
    const T ar = P.kp[i] * e - P.kd[i] * v[i];
    if (ar_out) ar_out[i] = val(ar);
    const T a = clampv(ar, -val(P.a_max), val(P.a_max));
    Fd[i] = P.m * (i == 2 ? a + P.g : a);
  }
  // collective thrust: desired force projected on the current body z axis
  T b3[3];
  body_z(q, b3);
  const T fc = Fd[0] * b3[0] + Fd[1] * b3[1] + Fd[2] * b3[2];
  // desired attitude: z along the desired force, x towards the heading
  const T nF = sqrt(Fd[0] * Fd[0] + Fd[1] * Fd[1] + Fd[2] * Fd[2]);
  const T zd[3] = {Fd[0] / nF, Fd[1] / nF, Fd[2] / nF};
  const T ch[3] = {T(std::cos(cmd[3])), T(std::sin(cmd[3])), T(0.0)};
  T yr[3];
  cross(zd, ch, yr);
  const T ny = sqrt(yr[0] * yr[0] + yr[1] * yr[1] + yr[2] * yr[2]);
  const T yd[3] = {yr[0] / ny, yr[1] / ny, yr[2] / ny};
  T xd[3];
  cross(yd, zd, xd);
  T Rd[3][3];
  for (int i = 0; i < 3; ++i) {
    Rd[i][0] = xd[i];
    Rd[i][1] = yd[i];
    Rd[i][2] = zd[i];
  }
  T qd[4];
  shepperd(Rd, qd);
  // attitude error q_e = q^* o q_d, shortest way round
  const T qc[4] = {q[0], -q[1], -q[2], -q[3]};
  T qe[4];
  hamilton(qc, qd, qe);
  if (val(qe[0]) < 0.0)
    for (int i = 0; i < 4; ++i) qe[i] = -qe[i];
  // attitude P -> desired body rates; rate P scaled by the axis torque limit
  T u[4];
  u[0] = fc;
  for (int i = 0; i < 3; ++i) {
    const T wdes = T(2.0) * P.katt[i] * qe[1 + i];
    if (e_out) e_out[i] = wdes - om[i];
    if (xi)
      u[1 + i] = T(F.taumax[i]) * (P.krate[i] * (wdes - om[i]) + P.kI[i] * xi[i] - P.kD[i] * wdot[i]);
    else
      u[1 + i] = P.krate[i] * T(F.taumax[i]) * (wdes - om[i]);
  }
  // inverse allocation, then per-rotor clamp in Omega^2 and square root
  const double om2max = val(P.omega_max) * val(P.omega_max);
  for (int i = 0; i < 4; ++i) {
    T fi = T(F.Ginv[i][0]) * u[0];
    for (int j = 1; j < 4; ++j) fi = fi + T(F.Ginv[i][j]) * u[j];
    const T S = fi / P.kt;
    if (S_out) S_out[i] = val(S);
    w[i] = sqrt(clampv(S, 0.0, om2max));
  }
}

// One classical RK4 step of length h of the 17 states with the rotor command
// w held (zero-order hold) over the four stages.
template <class T>
void rk4_core(const Group<T>& P, const Fixed& F, const T x[NX], const T w[4], double h, T xn[NX]) {
  T k1[NX], k2[NX], k3[NX], k4[NX], y[NX];
  derivative(P, F, x, w, k1);
  for (int i = 0; i < NX; ++i) y[i] = x[i] + T(0.5 * h) * k1[i];
  derivative(P, F, y, w, k2);
  for (int i = 0; i < NX; ++i) y[i] = x[i] + T(0.5 * h) * k2[i];
  derivative(P, F, y, w, k3);
  for (int i = 0; i < NX; ++i) y[i] = x[i] + T(h) * k3[i];
  derivative(P, F, y, w, k4);
  for (int i = 0; i < NX; ++i)
    xn[i] = x[i] + T(h / 6.0) * (k1[i] + T(2.0) * k2[i] + T(2.0) * k3[i] + k4[i]);
}

// One step, open or closed loop (P rate loop).  Open loop: cmd holds the
// rotor speed commands.
template <class T>
void rk4_step(const Group<T>& P, const Fixed& F, int mode, const T x[NX], const double cmd[4], double h,
              T xn[NX]) {
  T w[4];
  if (mode == CLOSED_LOOP) {
    controller(P, F, x, cmd, w);
  } else {
    for (int i = 0; i < 4; ++i) w[i] = T(cmd[i]);
  }
  rk4_core(P, F, x, w, h, xn);
}

// One step of the PID variant on the 20-state x = (17 states, xi): omega' at
// the step start from Eq. (qd4) (it does not depend on the rotor command), the
// controller, RK4 of the 17 states, then xi <- clamp(xi + h e, +-xi_max).
template <class T>
void rk4_step_pid(const Group<T>& P, const Fixed& F, const T x[NXP], const double cmd[4], double h, T xn[NXP]) {
  T d0[NX];
  derivative(P, F, x, x + 13, d0);
  T w[4], e[3];
  controller(P, F, x, cmd, w, nullptr, nullptr, x + NX, d0 + 10, e);
  rk4_core(P, F, x, w, h, xn);
  for (int i = 0; i < 3; ++i) {
    const double lim = val(P.xi_max[i]);
    xn[NX + i] = clampv(x[NX + i] + T(h) * e[i], -lim, lim);
  }
}

// Either step on a state of state_dim(mode) components.
template <class T>
void step_any(const Group<T>& P, const Fixed& F, int mode, const T* x, const double cmd[4], double h, T* xn) {
  if (mode == CLOSED_LOOP_PID)
    rk4_step_pid(P, F, x, cmd, h, xn);
  else
    rk4_step(P, F, mode, x, cmd, h, xn);
}

}  // namespace orc
