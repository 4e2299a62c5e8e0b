// Device models of the two other agent types that share the quadrotors'
// persistent launch (the paper's simulator runs fixed-wing drones, quadrotors
// and cars, Sec. III-B; it cites their models without equations):
//
//   car (type 1)         kinematic bicycle on the rear axle, pure pursuit
//                        towards the waypoint (kappa = 2 sin(alpha) /
//                        max(distance, l_min)): p' = v (c, s), v' = a,
//                        (c, s)' = v kappa (-s, c); inputs kappa (curvature,
//                        |kappa| <= tan(delta_max)/L_w) and a, held over the
//                        RK4 stages
//   fixed-wing (type 2)  coordinated-turn guidance model without wind:
//                        p' = V (c, s), h'' = -b_hd h' + b_h (h_c - h),
//                        V' = b_V (V_c - V), (c, s)' = (g tan(phi)/V)(-s, c),
//                        phi' = b_phi (phi_c - phi); phi_c from the course
//                        error to the waypoint, clamped to +-phi_max
//
// Both use components of the same 17-float planar state: p 0-2, speed 3,
// climb rate 5, heading unit vector 6-7, bank 10; the rest stay unchanged.
#pragma once
#include "model_fwd.cuh"

namespace qs {

enum { TYPE_QUAD = 0, TYPE_CAR = 1, TYPE_FIXED_WING = 2 };

// Car: curvature and acceleration for the command (x_c, y_c, -, v_c).
__device__ __forceinline__ void car_controller(const DevGroup& P, const float* x, const float4 c, float& kappa,
                                               float& a) {
  const float dx = c.x - x[0], dy = c.y - x[1];
  const float cross = x[6] * dy - x[7] * dx;  // |d| sin(alpha)
  const float d2 = dx * dx + dy * dy;
  const float kmax = P.vk[0];
  if (!(d2 > 0.f)) {
    kappa = 0.f;
  } else {
    const float dist = d2 * rsqrtf(d2);
    const float ld = fmaxf(dist, P.vk[3]);
    kappa = clampf(2.f * cross / (dist * ld), -kmax, kmax);
  }
  a = clampf(P.vk[2] * (c.w - x[3]), -P.vk[1], P.vk[1]);
}

// Fixed-wing: bank command for the command (x_c, y_c, h_c, V_c).
__device__ __forceinline__ float fw_controller(const DevGroup& P, const float* x, const float4 c) {
  const float dx = c.x - x[0], dy = c.y - x[1];
  const float ch = x[6], sh = x[7];
  const float cross = ch * dy - sh * dx, dot = ch * dx + sh * dy;
  const float err = (cross == 0.f && dot == 0.f) ? 0.f : atan2f(cross, dot);
  return clampf(P.vk[2] * err, -P.vk[1], P.vk[1]);
}

// One RK4 step of a car with the inputs held; components 0, 1, 3, 6, 7.
__device__ __forceinline__ void car_step(const DevGroup& P, St& x, const float4 c, const StepH& H) {
  float kappa, a;
  car_controller(P, x.a, c, kappa, a);
  const float px = x.a[0], py = x.a[1], v0 = x.a[3], c0 = x.a[6], s0 = x.a[7];
  float ap[5] = {0.f, 0.f, 0.f, 0.f, 0.f};  // RK4 sums of (p_x, p_y, v, c, s)
  float v = v0, cc = c0, ss = s0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float w = v * kappa;
    const float d[5] = {v * cc, v * ss, a, -ss * w, cc * w};
    const float wk = (k == 0 || k == 3) ? 1.f : 2.f;
#pragma unroll
    for (int j = 0; j < 5; ++j) ap[j] += wk * d[j];
    if (k < 3) {
      const float hk = k < 2 ? H.h2 : H.h;
      v = v0 + hk * d[2];
      cc = c0 + hk * d[3];
      ss = s0 + hk * d[4];
    }
  }
  x.a[0] = px + H.h6 * ap[0];
  x.a[1] = py + H.h6 * ap[1];
  x.a[3] = v0 + H.h6 * ap[2];
  x.a[6] = c0 + H.h6 * ap[3];
  x.a[7] = s0 + H.h6 * ap[4];
}

// One RK4 step of a fixed-wing drone with the commands held; components 0, 1,
// 2, 3, 5, 6, 7, 10.
__device__ __forceinline__ void fw_step(const DevGroup& P, St& x, const float4 c, const StepH& H) {
  const float phic = fw_controller(P, x.a, c);
  const float hc = c.z, Vc = c.w;
  const float bphi = P.vk[0], bhd = P.vk[3], bh = P.vk[4], bV = P.vk[5];
  enum { J = 8 };
  const int idx[J] = {0, 1, 2, 3, 5, 6, 7, 10};
  float y0[J], y[J], acc[J];
#pragma unroll
  for (int j = 0; j < J; ++j) { y0[j] = x.a[idx[j]]; y[j] = y0[j]; acc[j] = 0.f; }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    // y = (p_n, p_e, h, V, hdot, c, s, phi).  Course rate g tan(phi) / V by the
    // fast sine, cosine and divide: |phi| stays below phi_max < pi/2, where
    // they hold about 1e-6 relative, far inside the model's tolerances
    const float turn = P.g * __fdividef(__sinf(y[7]), __cosf(y[7]) * y[3]);
    const float d[J] = {y[3] * y[5], y[3] * y[6], y[4], bV * (Vc - y[3]), bhd * (0.f - y[4]) + bh * (hc - y[2]),
                        -y[6] * turn, y[5] * turn, bphi * (phic - y[7])};
    const float wk = (k == 0 || k == 3) ? 1.f : 2.f;
#pragma unroll
    for (int j = 0; j < J; ++j) acc[j] += wk * d[j];
    if (k < 3) {
      const float hk = k < 2 ? H.h2 : H.h;
#pragma unroll
      for (int j = 0; j < J; ++j) y[j] = y0[j] + hk * d[j];
    }
  }
#pragma unroll
  for (int j = 0; j < J; ++j) x.a[idx[j]] = y0[j] + H.h6 * acc[j];
}

__device__ __forceinline__ void vehicle_step(const DevGroup& P, St& x, const float4 c, const StepH& H) {
  if (P.vt == (float)TYPE_CAR)
    car_step(P, x, c, H);
  else
    fw_step(P, x, c, H);
}

}  // namespace qs
