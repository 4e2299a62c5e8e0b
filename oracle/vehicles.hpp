// TEST INFRASTRUCTURE ONLY: the plain FP64 definitions of the two other agent
// types the simulator runs beside the quadrotors.  Shares no code with the
// CUDA library.
//
// The paper lists three robot types implemented in its simulator --
// fixed-wing drones, quadrotors and cars (Sec. III-B, first paragraph) -- and
// cites the models of the first and the last without giving their equations.
// The readings taken here are the standard forms of the models it cites:
//
//   Car (type 1): kinematic bicycle, the low-speed form of a bicycle model,
//   on the rear-axle reference point, steered by pure pursuit towards the
//   waypoint.  State components used (of the 17): position p_x, p_y (0, 1),
//   height z (2, held), speed v (3), heading as a unit vector (c, s) =
//   (cos psi, sin psi) (6, 7).  Inputs u = (kappa, a), path curvature and
//   acceleration:
//       p_x' = v c,  p_y' = v s,  v' = a,  (c, s)' = v kappa (-s, c).
//   Controller (once per step, held over the RK4 stages), command =
//   (x_c, y_c, -, v_c): d = (x_c - p_x, y_c - p_y), kappa = 2 sin(alpha) /
//   max(|d|, l_min) with sin(alpha) = (c d_y - s d_x) / |d| (pure pursuit
//   aimed at the waypoint, for any bearing: continuous in the state),
//   |kappa| <= tan(delta_max) / L_w; a = clamp(k_v (v_c - v)).
//   veh = [L_w, tan(delta_max), a_max, k_v, l_min].
//
//   Fixed-wing (type 2): the point-mass guidance model of a fixed-wing drone
//   in coordinated flight without wind, with first-order autopilot loops on
//   bank and airspeed and a second-order altitude loop.  State components
//   used: p_n, p_e, h (0, 1, 2), airspeed V (3), climb rate h' (5), course as
//   a unit vector (c, s) (6, 7), bank phi (10).  Inputs u = (phi_c, h_c, V_c):
//       p_n' = V c,  p_e' = V s,  h' = hdot,  hdot' = b_hd (0 - hdot) + b_h (h_c - h),
//       V' = b_V (V_c - V),  (c, s)' = (g tan(phi) / V) (-s, c),
//       phi' = b_phi (phi_c - phi).
//   Controller, command = (x_c, y_c, h_c, V_c): course error chi_e =
//   atan2(c d_y - s d_x, c d_x + s d_y) to the waypoint, phi_c =
//   clamp(k_chi chi_e, +-phi_max).  veh = [b_phi, phi_max, k_chi, b_hd, b_h, b_V].
//
// Both types take the same RK4 step with the inputs held (as the quadrotor,
// Sec. III-B), run in the closed-loop mode only, and have no adjoint.
#pragma once
#include <cmath>
#include "quad_model.hpp"

namespace orc {

enum { TYPE_QUAD = 0, TYPE_CAR = 1, TYPE_FIXED_WING = 2 };

template <class T>
T clamp_sym(T x, double lim) {
  return clampv(x, -lim, lim);
}

// Inputs of a car or a fixed-wing drone at state x for its command.
template <class T>
void vehicle_controller(const Group<T>& P, const T x[NX], const double cmd[4], T u[3]) {
  const T dx = T(cmd[0]) - x[0], dy = T(cmd[1]) - x[1];
  const T c = x[6], s = x[7];
  const T cross = c * dy - s * dx;
  if (P.type == TYPE_CAR) {
    const double Lw = P.veh[0], kmax = P.veh[1] / Lw;
    const T dist = sqrt(dx * dx + dy * dy);
    T kappa = T(0.0);
    if (val(dist) > 0.0) {
      const T ld = val(dist) > P.veh[4] ? dist : T(P.veh[4]);
      kappa = clamp_sym(T(2.0) * cross / (dist * ld), kmax);
    }
    u[0] = kappa;
    u[1] = clamp_sym(T(P.veh[3]) * (T(cmd[3]) - x[3]), P.veh[2]);
    u[2] = T(0.0);
  } else {
    const T dot = c * dx + s * dy;
    const T err = (val(cross) == 0.0 && val(dot) == 0.0) ? T(0.0) : atan2(cross, dot);
    u[0] = clamp_sym(T(P.veh[2]) * err, P.veh[1]);
    u[1] = T(cmd[2]);
    u[2] = T(cmd[3]);
  }
}

// Time derivative of a car or fixed-wing state for held inputs u; the
// components a type does not use have derivative 0.
template <class T>
void vehicle_derivative(const Group<T>& P, const T x[NX], const T u[3], T dx[NX]) {
  for (int i = 0; i < NX; ++i) dx[i] = T(0.0);
  const T v = x[3], c = x[6], s = x[7];
  dx[0] = v * c;
  dx[1] = v * s;
  T turn;  // heading or course rate
  if (P.type == TYPE_CAR) {
    dx[3] = u[1];
    turn = v * u[0];
  } else {
    dx[2] = x[5];
    dx[5] = T(P.veh[3]) * (T(0.0) - x[5]) + T(P.veh[4]) * (u[1] - x[2]);
    dx[3] = T(P.veh[5]) * (u[2] - v);
    turn = P.g * tan(x[10]) / v;
    dx[10] = T(P.veh[0]) * (u[0] - x[10]);
  }
  dx[6] = -s * turn;
  dx[7] = c * turn;
}

// One RK4 step with the controller's inputs held over the four stages.
template <class T>
void vehicle_step(const Group<T>& P, const T x[NX], const double cmd[4], double h, T xn[NX]) {
  T u[3];
  vehicle_controller(P, x, cmd, u);
  T k1[NX], k2[NX], k3[NX], k4[NX], y[NX];
  vehicle_derivative(P, x, u, k1);
  for (int i = 0; i < NX; ++i) y[i] = x[i] + T(0.5 * h) * k1[i];
  vehicle_derivative(P, y, u, k2);
  for (int i = 0; i < NX; ++i) y[i] = x[i] + T(0.5 * h) * k2[i];
  vehicle_derivative(P, y, u, k3);
  for (int i = 0; i < NX; ++i) y[i] = x[i] + T(h) * k3[i];
  vehicle_derivative(P, y, u, k4);
  for (int i = 0; i < NX; ++i)
    xn[i] = x[i] + T(h / 6.0) * (k1[i] + T(2.0) * k2[i] + T(2.0) * k3[i] + k4[i]);
}

// One step of any agent: vehicles by their model, quadrotors by the mode.
template <class T>
void agent_step(const Group<T>& P, const Fixed& F, int mode, const T* x, const double cmd[4], double h, T* xn) {
  if (P.type != TYPE_QUAD)
    vehicle_step(P, x, cmd, h, xn);
  else
    step_any(P, F, mode, x, cmd, h, xn);
}

}  // namespace orc
