// Device model of one quadrotor step, one thread per agent, FP32 in registers.
//
//   derivative   Eq. (qd1)-(qd4), Eq. (2), Eq. (3) of arXiv 2308.12698 Sec. III-B,
//                plus first-order rotor lag and linear drag
//   controller   cascaded position PD -> attitude P -> normalised rate P ->
//                G^-1 -> rotor clamp (the paper's inner body-rate loop,
//                Sec. III-B, completed as documented in quadsim.h)
//   rk4          classical RK4, command held over the stages (Sec. III-B)
//   *_vjp        hand-written vector-Jacobian products of the above for the
//                discrete adjoint
//
// State vector index map (17 floats): p 0-2, v 3-5, q 6-9 (w x y z),
// omega 10-12, Omega 13-16.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace qs {

enum { PX = 0, VX = 3, QW = 6, QX = 7, QY = 8, QZ = 9, WX = 10, OM = 13, NX = 17 };
enum { TH_KP = 0, TH_KD = 3, TH_KATT = 6, TH_KRATE = 9, TH_M = 12, TH_J = 13, NTH = 16 };

// Per-group constants, derived on the host in double from the public
// parameters and rounded once to float.  44 floats, float4-aligned rows.
struct __align__(16) DevGroup {
  float m, inv_m, g, cd_m;        // mass, 1/m, gravity, c_d/m
  float Jx, Jy, Jz, inv_tau;      // principal inertias, 1/tau_m
  float iJx, iJy, iJz, om2max;    // 1/J, omega_max^2
  float gx, gy, gz, c_d;          // (Jy-Jz)/Jx, (Jz-Jx)/Jy, (Jx-Jy)/Jz, drag
  float kf, kfLs, kfLc, km;       // kt, kt L sin(a), kt L cos(a), kq
  float kp[3], a_max;
  float kd[3], mix0;              // mix0 = 1/(4 kt)
  float katt2[3], mix1;           // 2 katt; mix1 = 1/(4 kt L sin a)
  float krt[3], mix2;             // krate*taumax; mix2 = 1/(4 kt L cos a)
  float krate[3], mix3;           // mix3 = 1/(4 kq)
  float taumax[3], pad;
};
static_assert(sizeof(DevGroup) == 44 * 4, "DevGroup layout");

struct St {
  float a[NX];
};

// ------------------------------------------------------------ planar I/O --
// Plane k (0..3) holds float4 of components 4k..4k+3, plane 4 component 16.
__device__ __forceinline__ void load_state(const float* __restrict__ base, int64_t n, int64_t i, St& x) {
  const float4* P = reinterpret_cast<const float4*>(base);
  const float4 a = P[i], b = P[n + i], c = P[2 * n + i], d = P[3 * n + i];
  const float e = base[16 * n + i];
  x.a[0] = a.x; x.a[1] = a.y; x.a[2] = a.z; x.a[3] = a.w;
  x.a[4] = b.x; x.a[5] = b.y; x.a[6] = b.z; x.a[7] = b.w;
  x.a[8] = c.x; x.a[9] = c.y; x.a[10] = c.z; x.a[11] = c.w;
  x.a[12] = d.x; x.a[13] = d.y; x.a[14] = d.z; x.a[15] = d.w;
  x.a[16] = e;
}

__device__ __forceinline__ void store_state(float* __restrict__ base, int64_t n, int64_t i, const St& x) {
  float4* P = reinterpret_cast<float4*>(base);
  P[i] = make_float4(x.a[0], x.a[1], x.a[2], x.a[3]);
  P[n + i] = make_float4(x.a[4], x.a[5], x.a[6], x.a[7]);
  P[2 * n + i] = make_float4(x.a[8], x.a[9], x.a[10], x.a[11]);
  P[3 * n + i] = make_float4(x.a[12], x.a[13], x.a[14], x.a[15]);
  base[16 * n + i] = x.a[16];
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// Body z axis in the inertial frame: third column of R(q).
__device__ __forceinline__ void body_z(const St& x, float& bx, float& by, float& bz) {
  const float w = x.a[QW], qx = x.a[QX], qy = x.a[QY], qz = x.a[QZ];
  bx = 2.f * (qx * qz + w * qy);
  by = 2.f * (qy * qz - w * qx);
  bz = 1.f - 2.f * (qx * qx + qy * qy);
}

// --------------------------------------------------------- the derivative --
__device__ __forceinline__ void derivative(const DevGroup& P, const St& y, const float u[4], St& d) {
  const float s1 = y.a[OM] * y.a[OM], s2 = y.a[OM + 1] * y.a[OM + 1];
  const float s3 = y.a[OM + 2] * y.a[OM + 2], s4 = y.a[OM + 3] * y.a[OM + 3];
  // Eq. (2)-(3): collective thrust and body torques from the lagged rotor speeds
  const float fc = P.kf * ((s1 + s2) + (s3 + s4));
  const float tx = P.kfLs * ((s1 - s2) + (s4 - s3));
  const float ty = P.kfLc * ((s3 + s4) - (s1 + s2));
  const float tz = P.km * ((s1 - s2) + (s3 - s4));
  float bx, by, bz;
  body_z(y, bx, by, bz);
  const float T = fc * P.inv_m;
  // Eq. (qd1)
  d.a[0] = y.a[VX]; d.a[1] = y.a[VX + 1]; d.a[2] = y.a[VX + 2];
  // Eq. (qd2) with linear drag
  d.a[3] = bx * T - P.cd_m * y.a[VX];
  d.a[4] = by * T - P.cd_m * y.a[VX + 1];
  d.a[5] = bz * T - P.cd_m * y.a[VX + 2] - P.g;
  // Eq. (qd3): 1/2 q o [0, omega]
  const float w = y.a[QW], qx = y.a[QX], qy = y.a[QY], qz = y.a[QZ];
  const float wx = y.a[WX], wy = y.a[WX + 1], wz = y.a[WX + 2];
  d.a[QW] = 0.5f * (-qx * wx - qy * wy - qz * wz);
  d.a[QX] = 0.5f * (w * wx + qy * wz - qz * wy);
  d.a[QY] = 0.5f * (w * wy + qz * wx - qx * wz);
  d.a[QZ] = 0.5f * (w * wz + qx * wy - qy * wx);
  // Eq. (qd4): omega' = I^-1 (tau - omega x I omega), diagonal I
  d.a[WX] = P.gx * (wy * wz) + tx * P.iJx;
  d.a[WX + 1] = P.gy * (wz * wx) + ty * P.iJy;
  d.a[WX + 2] = P.gz * (wx * wy) + tz * P.iJz;
  // rotor lag
#pragma unroll
  for (int i = 0; i < 4; ++i) d.a[OM + i] = (u[i] - y.a[OM + i]) * P.inv_tau;
}

// ---------------------------------------------------------- the controller --
// Forward intermediates shared by the controller and its VJP.
struct Ctl {
  float e[3], a[3];
  bool pass[3];          // acceleration clamp passes the gradient
  float F[3], b3[3], fc;
  float rn, zd[3];
  float ry, yd[3], xd[3];
  int branch;            // Shepperd branch 0:w 1:x 2:y 3:z
  float k;               // 0.5 / sqrt(t) of the branch
  float qd[4];
  float sgn;             // sign that makes qe.w >= 0
  float qe[4];           // after the sign fix
  float wd[3];
  float S[4];            // Omega^2 demanded by the mixer, before the clamp
};

__device__ __forceinline__ void controller_fwd(const DevGroup& P, const St& x, const float4 c, float ch, float sh,
                                               Ctl& C, float u[4]) {
  const float cc[3] = {c.x, c.y, c.z};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    C.e[i] = cc[i] - x.a[PX + i];
    const float ar = P.kp[i] * C.e[i] - P.kd[i] * x.a[VX + i];
    C.pass[i] = (ar >= -P.a_max) && (ar <= P.a_max);
    C.a[i] = clampf(ar, -P.a_max, P.a_max);
  }
  C.F[0] = P.m * C.a[0];
  C.F[1] = P.m * C.a[1];
  C.F[2] = P.m * (C.a[2] + P.g);
  body_z(x, C.b3[0], C.b3[1], C.b3[2]);
  C.fc = C.F[0] * C.b3[0] + C.F[1] * C.b3[1] + C.F[2] * C.b3[2];
  // desired body z along the force, body y from the heading, x = y cross z
  C.rn = rsqrtf(C.F[0] * C.F[0] + C.F[1] * C.F[1] + C.F[2] * C.F[2]);
  C.zd[0] = C.F[0] * C.rn; C.zd[1] = C.F[1] * C.rn; C.zd[2] = C.F[2] * C.rn;
  const float yr0 = -C.zd[2] * sh, yr1 = C.zd[2] * ch, yr2 = C.zd[0] * sh - C.zd[1] * ch;
  C.ry = rsqrtf(yr0 * yr0 + yr1 * yr1 + yr2 * yr2);
  C.yd[0] = yr0 * C.ry; C.yd[1] = yr1 * C.ry; C.yd[2] = yr2 * C.ry;
  C.xd[0] = C.yd[1] * C.zd[2] - C.yd[2] * C.zd[1];
  C.xd[1] = C.yd[2] * C.zd[0] - C.yd[0] * C.zd[2];
  C.xd[2] = C.yd[0] * C.zd[1] - C.yd[1] * C.zd[0];
  // R_des columns xd, yd, zd:  R[r][0] = xd[r], R[r][1] = yd[r], R[r][2] = zd[r]
  const float R00 = C.xd[0], R10 = C.xd[1], R20 = C.xd[2];
  const float R01 = C.yd[0], R11 = C.yd[1], R21 = C.yd[2];
  const float R02 = C.zd[0], R12 = C.zd[1], R22 = C.zd[2];
  // Shepperd: scalar branch if trace > 0, else the largest diagonal
  const float tr = R00 + R11 + R22;
  int br = 0;
  if (!(tr > 0.f)) {
    br = 1;
    if (R11 > R00) br = 2;
    if (R22 > (br == 2 ? R11 : R00)) br = 3;
  }
  C.branch = br;
  float t;
  if (br == 0) t = 1.f + tr;
  else if (br == 1) t = 1.f + R00 - R11 - R22;
  else if (br == 2) t = 1.f - R00 + R11 - R22;
  else t = 1.f - R00 - R11 + R22;
  const float rs = rsqrtf(t);  // t >= 1 on the branch taken
  const float r = t * rs;
  C.k = 0.5f * rs;
  if (br == 0) {
    C.qd[0] = 0.5f * r; C.qd[1] = (R21 - R12) * C.k; C.qd[2] = (R02 - R20) * C.k; C.qd[3] = (R10 - R01) * C.k;
  } else if (br == 1) {
    C.qd[1] = 0.5f * r; C.qd[0] = (R21 - R12) * C.k; C.qd[2] = (R01 + R10) * C.k; C.qd[3] = (R02 + R20) * C.k;
  } else if (br == 2) {
    C.qd[2] = 0.5f * r; C.qd[0] = (R02 - R20) * C.k; C.qd[1] = (R01 + R10) * C.k; C.qd[3] = (R12 + R21) * C.k;
  } else {
    C.qd[3] = 0.5f * r; C.qd[0] = (R10 - R01) * C.k; C.qd[1] = (R02 + R20) * C.k; C.qd[2] = (R12 + R21) * C.k;
  }
  // q_e = conj(q) o q_d
  const float w = x.a[QW], qx = x.a[QX], qy = x.a[QY], qz = x.a[QZ];
  const float dw = C.qd[0], dx = C.qd[1], dy = C.qd[2], dz = C.qd[3];
  float ew = w * dw + qx * dx + qy * dy + qz * dz;
  float ex = w * dx - dw * qx - qy * dz + qz * dy;
  float ey = w * dy - dw * qy - qz * dx + qx * dz;
  float ez = w * dz - dw * qz - qx * dy + qy * dx;
  C.sgn = ew < 0.f ? -1.f : 1.f;
  C.qe[0] = C.sgn * ew; C.qe[1] = C.sgn * ex; C.qe[2] = C.sgn * ey; C.qe[3] = C.sgn * ez;
  // attitude P, then rate P scaled by the axis torque limit
  float tau[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    C.wd[i] = P.katt2[i] * C.qe[1 + i];
    tau[i] = P.krt[i] * (C.wd[i] - x.a[WX + i]);
  }
  // G^-1 by the orthogonal rows of G, in Omega^2 units
  const float f0 = P.mix0 * C.fc, f1 = P.mix1 * tau[0], f2 = P.mix2 * tau[1], f3 = P.mix3 * tau[2];
  C.S[0] = (f0 + f1) + (f3 - f2);
  C.S[1] = (f0 - f1) - (f2 + f3);
  C.S[2] = (f0 - f1) + (f2 + f3);
  C.S[3] = (f0 + f1) + (f2 - f3);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float s = clampf(C.S[i], 0.f, P.om2max);
    u[i] = s > 0.f ? s * rsqrtf(s) : 0.f;
  }
}

__device__ __forceinline__ void controller(const DevGroup& P, const St& x, const float4 c, float ch, float sh,
                                           float u[4]) {
  Ctl C;
  controller_fwd(P, x, c, ch, sh, C, u);
}

// ------------------------------------------------------------------ RK4 --
struct StepH {
  float h, h2, h6;  // h, h/2, h/6 (rounded once on the host)
};

__device__ __forceinline__ void rk4(const DevGroup& P, St& x, const float u[4], const StepH& H) {
  St k, y, acc;
  derivative(P, x, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) { acc.a[i] = k.a[i]; y.a[i] = x.a[i] + H.h2 * k.a[i]; }
  derivative(P, y, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) { acc.a[i] += 2.f * k.a[i]; y.a[i] = x.a[i] + H.h2 * k.a[i]; }
  derivative(P, y, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) { acc.a[i] += 2.f * k.a[i]; y.a[i] = x.a[i] + H.h * k.a[i]; }
  derivative(P, y, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) { acc.a[i] += k.a[i]; x.a[i] = x.a[i] + H.h6 * acc.a[i]; }
}

template <int MODE>
__device__ __forceinline__ void step(const DevGroup& P, St& x, const float4 c, float ch, float sh, const StepH& H) {
  float u[4];
  if (MODE == 1) {
    controller(P, x, c, ch, sh, u);
  } else {
    u[0] = c.x; u[1] = c.y; u[2] = c.z; u[3] = c.w;
  }
  rk4(P, x, u, H);
}

// ------------------------------------------------------------------ VJPs --
// Accumulates into yb (state cotangent), ub (rotor command cotangent) and
// tb (theta cotangent) the products of g with the Jacobians of derivative().
__device__ __forceinline__ void derivative_vjp(const DevGroup& P, const St& y, const St& g, St& yb, float ub[4],
                                               float tb[NTH]) {
  const float O1 = y.a[OM], O2 = y.a[OM + 1], O3 = y.a[OM + 2], O4 = y.a[OM + 3];
  const float s1 = O1 * O1, s2 = O2 * O2, s3 = O3 * O3, s4 = O4 * O4;
  const float fc = P.kf * ((s1 + s2) + (s3 + s4));
  const float tx = P.kfLs * ((s1 - s2) + (s4 - s3));
  const float ty = P.kfLc * ((s3 + s4) - (s1 + s2));
  const float tz = P.km * ((s1 - s2) + (s3 - s4));
  const float w = y.a[QW], qx = y.a[QX], qy = y.a[QY], qz = y.a[QZ];
  const float wx = y.a[WX], wy = y.a[WX + 1], wz = y.a[WX + 2];
  float bx, by, bz;
  body_z(y, bx, by, bz);
  const float T = fc * P.inv_m;
  const float gvx = g.a[3], gvy = g.a[4], gvz = g.a[5];
  // p' = v
  yb.a[VX] += g.a[0]; yb.a[VX + 1] += g.a[1]; yb.a[VX + 2] += g.a[2];
  // v' = b3 T - cd_m v - g e3
  yb.a[VX] -= P.cd_m * gvx; yb.a[VX + 1] -= P.cd_m * gvy; yb.a[VX + 2] -= P.cd_m * gvz;
  const float Tb = gvx * bx + gvy * by + gvz * bz;
  const float fcb = Tb * P.inv_m;
  const float gv_v = gvx * y.a[VX] + gvy * y.a[VX + 1] + gvz * y.a[VX + 2];
  tb[TH_M] += -Tb * T * P.inv_m + gv_v * P.cd_m * P.inv_m;
  const float bbx = gvx * T, bby = gvy * T, bbz = gvz * T;
  float qbw = 2.f * (qy * bbx - qx * bby);
  float qbx = 2.f * (qz * bbx - w * bby) - 4.f * qx * bbz;
  float qby = 2.f * (w * bbx + qz * bby) - 4.f * qy * bbz;
  float qbz = 2.f * (qx * bbx + qy * bby);
  // q' = 1/2 q o [0, omega]
  const float gw = 0.5f * g.a[QW], gx = 0.5f * g.a[QX], gy = 0.5f * g.a[QY], gz = 0.5f * g.a[QZ];
  qbw += gx * wx + gy * wy + gz * wz;
  qbx += -gw * wx - gy * wz + gz * wy;
  qby += -gw * wy + gx * wz - gz * wx;
  qbz += -gw * wz - gx * wy + gy * wx;
  yb.a[QW] += qbw; yb.a[QX] += qbx; yb.a[QY] += qby; yb.a[QZ] += qbz;
  float wbx = -gw * qx + gx * w + gy * qz - gz * qy;
  float wby = -gw * qy - gx * qz + gy * w + gz * qx;
  float wbz = -gw * qz + gx * qy - gy * qx + gz * w;
  // omega'_x = ((Jy - Jz) wy wz + tx) / Jx, and cyclic
  const float nbx = g.a[WX] * P.iJx, nby = g.a[WX + 1] * P.iJy, nbz = g.a[WX + 2] * P.iJz;
  const float cx = P.Jy - P.Jz, cy = P.Jz - P.Jx, cz = P.Jx - P.Jy;
  const float dwx = (cx * (wy * wz) + tx) * P.iJx;
  const float dwy = (cy * (wz * wx) + ty) * P.iJy;
  const float dwz = (cz * (wx * wy) + tz) * P.iJz;
  tb[TH_J] += -nbx * dwx - nby * (wz * wx) + nbz * (wx * wy);
  tb[TH_J + 1] += nbx * (wy * wz) - nby * dwy - nbz * (wx * wy);
  tb[TH_J + 2] += -nbx * (wy * wz) + nby * (wz * wx) - nbz * dwz;
  wbx += nby * cy * wz + nbz * cz * wy;
  wby += nbx * cx * wz + nbz * cz * wx;
  wbz += nbx * cx * wy + nby * cy * wx;
  yb.a[WX] += wbx; yb.a[WX + 1] += wby; yb.a[WX + 2] += wbz;
  // rotors: thrust/torque rows of G on s_i = Omega_i^2, then the lag
  const float a0 = P.kf * fcb, a1 = P.kfLs * nbx, a2 = P.kfLc * nby, a3 = P.km * nbz;
  const float sb1 = (a0 + a1) + (a3 - a2);
  const float sb2 = (a0 - a1) - (a2 + a3);
  const float sb3 = (a0 - a1) + (a2 + a3);
  const float sb4 = (a0 + a1) + (a2 - a3);
  const float gO1 = g.a[OM] * P.inv_tau, gO2 = g.a[OM + 1] * P.inv_tau;
  const float gO3 = g.a[OM + 2] * P.inv_tau, gO4 = g.a[OM + 3] * P.inv_tau;
  yb.a[OM] += 2.f * O1 * sb1 - gO1;
  yb.a[OM + 1] += 2.f * O2 * sb2 - gO2;
  yb.a[OM + 2] += 2.f * O3 * sb3 - gO3;
  yb.a[OM + 3] += 2.f * O4 * sb4 - gO4;
  ub[0] += gO1; ub[1] += gO2; ub[2] += gO3; ub[3] += gO4;
}

// Cotangent of the controller: ub (rotor commands) -> xb (state), tb (theta).
__device__ __forceinline__ void controller_vjp(const DevGroup& P, const St& x, const float4 c, float ch, float sh,
                                               const float ub[4], St& xb, float tb[NTH]) {
  Ctl C;
  float u[4];
  controller_fwd(P, x, c, ch, sh, C, u);
  // sqrt(clamp(S)): gradient passes on 0 < S <= om2max (sqrt'(0) taken as 0)
  float Sb[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float s = C.S[i];
    Sb[i] = (s > 0.f && s <= P.om2max) ? ub[i] * 0.5f * rsqrtf(s) : 0.f;
  }
  const float fcb = P.mix0 * ((Sb[0] + Sb[1]) + (Sb[2] + Sb[3]));
  float taub[3];
  taub[0] = P.mix1 * ((Sb[0] - Sb[1]) + (Sb[3] - Sb[2]));
  taub[1] = P.mix2 * ((Sb[2] + Sb[3]) - (Sb[0] + Sb[1]));
  taub[2] = P.mix3 * ((Sb[0] - Sb[1]) + (Sb[2] - Sb[3]));
  // tau = krate taumax (wd - omega), wd = 2 katt qe
  float qeb[4];
  qeb[0] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float err = C.wd[i] - x.a[WX + i];
    tb[TH_KRATE + i] += taub[i] * P.taumax[i] * err;
    const float wdb = taub[i] * P.krt[i];
    xb.a[WX + i] -= wdb;
    tb[TH_KATT + i] += wdb * 2.f * C.qe[1 + i];
    qeb[1 + i] = wdb * P.katt2[i] * C.sgn;  // through the sign fix
  }
  // qe = conj(q) o qd
  const float w = x.a[QW], qx = x.a[QX], qy = x.a[QY], qz = x.a[QZ];
  const float dw = C.qd[0], dx = C.qd[1], dy = C.qd[2], dz = C.qd[3];
  const float Ew = qeb[0], Ex = qeb[1], Ey = qeb[2], Ez = qeb[3];
  xb.a[QW] += Ew * dw + Ex * dx + Ey * dy + Ez * dz;
  xb.a[QX] += Ew * dx - Ex * dw + Ey * dz - Ez * dy;
  xb.a[QY] += Ew * dy - Ex * dz - Ey * dw + Ez * dx;
  xb.a[QZ] += Ew * dz + Ex * dy - Ey * dx - Ez * dw;
  float qdb[4];
  qdb[0] = Ew * w - Ex * qx - Ey * qy - Ez * qz;
  qdb[1] = Ew * qx + Ex * w - Ey * qz + Ez * qy;
  qdb[2] = Ew * qy + Ex * qz + Ey * w - Ez * qx;
  qdb[3] = Ew * qz - Ex * qy + Ey * qx + Ez * w;
  // Shepperd, branch taken
  float Rb[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  const float R10 = C.xd[1], R20 = C.xd[2];
  const float R01 = C.yd[0], R21 = C.yd[2];
  const float R02 = C.zd[0], R12 = C.zd[1];
  const float k = C.k, k2x2 = 2.f * C.k * C.k;
  if (C.branch == 0) {
    const float kb = qdb[1] * (R21 - R12) + qdb[2] * (R02 - R20) + qdb[3] * (R10 - R01);
    Rb[2][1] += qdb[1] * k; Rb[1][2] -= qdb[1] * k;
    Rb[0][2] += qdb[2] * k; Rb[2][0] -= qdb[2] * k;
    Rb[1][0] += qdb[3] * k; Rb[0][1] -= qdb[3] * k;
    const float tb_ = (0.5f * qdb[0] - k2x2 * kb) * k;
    Rb[0][0] += tb_; Rb[1][1] += tb_; Rb[2][2] += tb_;
  } else if (C.branch == 1) {
    const float kb = qdb[0] * (R21 - R12) + qdb[2] * (R01 + R10) + qdb[3] * (R02 + R20);
    Rb[2][1] += qdb[0] * k; Rb[1][2] -= qdb[0] * k;
    Rb[0][1] += qdb[2] * k; Rb[1][0] += qdb[2] * k;
    Rb[0][2] += qdb[3] * k; Rb[2][0] += qdb[3] * k;
    const float tb_ = (0.5f * qdb[1] - k2x2 * kb) * k;
    Rb[0][0] += tb_; Rb[1][1] -= tb_; Rb[2][2] -= tb_;
  } else if (C.branch == 2) {
    const float kb = qdb[0] * (R02 - R20) + qdb[1] * (R01 + R10) + qdb[3] * (R12 + R21);
    Rb[0][2] += qdb[0] * k; Rb[2][0] -= qdb[0] * k;
    Rb[0][1] += qdb[1] * k; Rb[1][0] += qdb[1] * k;
    Rb[1][2] += qdb[3] * k; Rb[2][1] += qdb[3] * k;
    const float tb_ = (0.5f * qdb[2] - k2x2 * kb) * k;
    Rb[0][0] -= tb_; Rb[1][1] += tb_; Rb[2][2] -= tb_;
  } else {
    const float kb = qdb[0] * (R10 - R01) + qdb[1] * (R02 + R20) + qdb[2] * (R12 + R21);
    Rb[1][0] += qdb[0] * k; Rb[0][1] -= qdb[0] * k;
    Rb[0][2] += qdb[1] * k; Rb[2][0] += qdb[1] * k;
    Rb[1][2] += qdb[2] * k; Rb[2][1] += qdb[2] * k;
    const float tb_ = (0.5f * qdb[3] - k2x2 * kb) * k;
    Rb[0][0] -= tb_; Rb[1][1] -= tb_; Rb[2][2] += tb_;
  }
  // columns of R_des
  float xdb[3] = {Rb[0][0], Rb[1][0], Rb[2][0]};
  float ydb[3] = {Rb[0][1], Rb[1][1], Rb[2][1]};
  float zdb[3] = {Rb[0][2], Rb[1][2], Rb[2][2]};
  // xd = yd x zd
  ydb[0] += C.zd[1] * xdb[2] - C.zd[2] * xdb[1];
  ydb[1] += C.zd[2] * xdb[0] - C.zd[0] * xdb[2];
  ydb[2] += C.zd[0] * xdb[1] - C.zd[1] * xdb[0];
  zdb[0] += xdb[1] * C.yd[2] - xdb[2] * C.yd[1];
  zdb[1] += xdb[2] * C.yd[0] - xdb[0] * C.yd[2];
  zdb[2] += xdb[0] * C.yd[1] - xdb[1] * C.yd[0];
  // yd = yr / |yr|
  const float yy = C.yd[0] * ydb[0] + C.yd[1] * ydb[1] + C.yd[2] * ydb[2];
  const float yrb0 = (ydb[0] - C.yd[0] * yy) * C.ry;
  const float yrb1 = (ydb[1] - C.yd[1] * yy) * C.ry;
  const float yrb2 = (ydb[2] - C.yd[2] * yy) * C.ry;
  // yr = zd x (ch, sh, 0):  zdb += (ch, sh, 0) x yrb
  zdb[0] += sh * yrb2;
  zdb[1] += -ch * yrb2;
  zdb[2] += ch * yrb1 - sh * yrb0;
  // zd = F / |F|
  const float zz = C.zd[0] * zdb[0] + C.zd[1] * zdb[1] + C.zd[2] * zdb[2];
  float Fb[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Fb[i] = (zdb[i] - C.zd[i] * zz) * C.rn + fcb * C.b3[i];
  // fc = F . b3  ->  b3 -> q
  const float bbx = fcb * C.F[0], bby = fcb * C.F[1], bbz = fcb * C.F[2];
  xb.a[QW] += 2.f * (qy * bbx - qx * bby);
  xb.a[QX] += 2.f * (qz * bbx - w * bby) - 4.f * qx * bbz;
  xb.a[QY] += 2.f * (w * bbx + qz * bby) - 4.f * qy * bbz;
  xb.a[QZ] += 2.f * (qx * bbx + qy * bby);
  // F = m (a + g e3)
  tb[TH_M] += Fb[0] * C.a[0] + Fb[1] * C.a[1] + Fb[2] * (C.a[2] + P.g);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float arb = C.pass[i] ? P.m * Fb[i] : 0.f;
    tb[TH_KP + i] += arb * C.e[i];
    tb[TH_KD + i] -= arb * x.a[VX + i];
    xb.a[PX + i] -= P.kp[i] * arb;
    xb.a[VX + i] -= P.kd[i] * arb;
  }
}

// Adjoint of one RK4 step x_n -> x_{n+1}: lam <- (d x_{n+1} / d x_n)^T lam,
// tb += (d x_{n+1} / d theta)^T lam.  x is the step-start state.
template <int MODE>
__device__ __forceinline__ void step_vjp(const DevGroup& P, const St& x, const float4 c, float ch, float sh,
                                         const StepH& H, St& lam, float tb[NTH]) {
  float u[4];
  if (MODE == 1) {
    controller(P, x, c, ch, sh, u);
  } else {
    u[0] = c.x; u[1] = c.y; u[2] = c.z; u[3] = c.w;
  }
  St k, y2, y3, y4;
  derivative(P, x, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) y2.a[i] = x.a[i] + H.h2 * k.a[i];
  derivative(P, y2, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) y3.a[i] = x.a[i] + H.h2 * k.a[i];
  derivative(P, y3, u, k);
#pragma unroll
  for (int i = 0; i < NX; ++i) y4.a[i] = x.a[i] + H.h * k.a[i];
  const float h3 = 2.f * H.h6;
  float ub[4] = {0.f, 0.f, 0.f, 0.f};
  St xb = lam, g, yb;
  // k4 at y4 = x + h k3
#pragma unroll
  for (int i = 0; i < NX; ++i) { g.a[i] = H.h6 * lam.a[i]; yb.a[i] = 0.f; }
  derivative_vjp(P, y4, g, yb, ub, tb);
  // k3 at y3 = x + h/2 k2
#pragma unroll
  for (int i = 0; i < NX; ++i) { xb.a[i] += yb.a[i]; g.a[i] = h3 * lam.a[i] + H.h * yb.a[i]; yb.a[i] = 0.f; }
  derivative_vjp(P, y3, g, yb, ub, tb);
  // k2 at y2 = x + h/2 k1
#pragma unroll
  for (int i = 0; i < NX; ++i) { xb.a[i] += yb.a[i]; g.a[i] = h3 * lam.a[i] + H.h2 * yb.a[i]; yb.a[i] = 0.f; }
  derivative_vjp(P, y2, g, yb, ub, tb);
  // k1 at x
#pragma unroll
  for (int i = 0; i < NX; ++i) { xb.a[i] += yb.a[i]; g.a[i] = H.h6 * lam.a[i] + H.h2 * yb.a[i]; yb.a[i] = 0.f; }
  derivative_vjp(P, x, g, yb, ub, tb);
#pragma unroll
  for (int i = 0; i < NX; ++i) xb.a[i] += yb.a[i];
  if (MODE == 1) controller_vjp(P, x, c, ch, sh, ub, xb, tb);
  lam = xb;
}

}  // namespace qs
