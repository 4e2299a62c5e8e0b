// Hand-written vector-Jacobian products of the device model (model_fwd.cuh)
// for the discrete adjoint of the RK4 rollout: rb_derivative_vjp,
// controller_vjp and step_vjp (P and PID rate loops).  Subgradients: clamps pass the gradient on
// their closed interval, sqrt has derivative 0 at 0, branch choices (the roll
// half-angle formula, sign of q_e.w) are constants.
//
// The mass and the inertias enter the dynamics only through the derived
// group constants T2c = 2 kt / m, cd_m = c_d / m, gx, gy, gz (the gyroscopic
// coefficients) and txc, tyc, tzc (torque / inertia).  The sweep accumulates
// the cotangents of those eight constants (dc) and theta_from_derived turns
// them into m and J cotangents once per agent.

#pragma once
#include "model_fwd.cuh"

namespace qs {

// ------------------------------------------------------------------ VJPs --
// Cotangents of the derived dynamics constants of DevGroup, in this order:
// T2c, cd_m, gx, gy, gz, txc, tyc, tzc.
enum { DC_T2 = 0, DC_CD, DC_GX, DC_GY, DC_GZ, DC_TX, DC_TY, DC_TZ, NDC };

// Adds to yb (13) and dc (the derived constants), and writes to Omb (the
// stage's rotor speeds, 4), the products of g (13) with the Jacobians of
// rb_derivative at (y, Om).
__device__ __forceinline__ void rb_derivative_vjp(const DevGroup& P, const float* y, const float Om[4], const float* g,
                                                  float* yb, float Omb[4], float dc[NDC]) {
  const float s1 = Om[0] * Om[0], s2 = Om[1] * Om[1], s3 = Om[2] * Om[2], s4 = Om[3] * Om[3];
  const float Ssum = (s1 + s2) + (s3 + s4);
  const float T2 = P.T2c * Ssum;
  const float Dx = (s1 - s2) + (s4 - s3), Dy = (s3 + s4) - (s1 + s2), Dz = (s1 - s2) + (s3 - s4);
  const float w = y[QW], qx = y[QX], qy = y[QY], qz = y[QZ];
  const float wx = y[WX], wy = y[WX + 1], wz = y[WX + 2];
  const float bx = qx * qz + w * qy, by = qy * qz - w * qx, bxy = qx * qx + qy * qy;
  const float gvx = g[3], gvy = g[4], gvz = g[5];
  // p' = v ; v' = T2 (bx, by, 1/2 - bxy) - cd_m v - g e3
  yb[VX] += g[0] - P.cd_m * gvx;
  yb[VX + 1] += g[1] - P.cd_m * gvy;
  yb[VX + 2] += g[2] - P.cd_m * gvz;
  const float T2b = gvx * bx + gvy * by + gvz * (0.5f - bxy);
  dc[DC_T2] += T2b * Ssum;  // T2 = T2c * Ssum
  dc[DC_CD] -= gvx * y[VX] + gvy * y[VX + 1] + gvz * y[VX + 2];
  const float bbx = gvx * T2, bby = gvy * T2, bbxy = -gvz * T2;
  float qbw = qy * bbx - qx * bby;
  float qbx = qz * bbx - w * bby + 2.f * qx * bbxy;
  float qby = w * bbx + qz * bby + 2.f * qy * bbxy;
  float qbz = qx * bbx + qy * bby;
  // 2 q' = q o [0, omega]
  const float gw = g[QW], gx = g[QX], gy = g[QY], gz = g[QZ];
  qbw += gx * wx + gy * wy + gz * wz;
  qbx += -gw * wx - gy * wz + gz * wy;
  qby += -gw * wy + gx * wz - gz * wx;
  qbz += -gw * wz - gx * wy + gy * wx;
  yb[QW] += qbw; yb[QX] += qbx; yb[QY] += qby; yb[QZ] += qbz;
  float wbx = -gw * qx + gx * w + gy * qz - gz * qy;
  float wby = -gw * qy - gx * qz + gy * w + gz * qx;
  float wbz = -gw * qz + gx * qy - gy * qx + gz * w;
  // omega'_x = gx wy wz + txc Dx, and cyclic
  const float nx = g[WX], ny = g[WX + 1], nz = g[WX + 2];
  dc[DC_GX] += nx * (wy * wz);
  dc[DC_GY] += ny * (wz * wx);
  dc[DC_GZ] += nz * (wx * wy);
  dc[DC_TX] += nx * Dx;
  dc[DC_TY] += ny * Dy;
  dc[DC_TZ] += nz * Dz;
  wbx += ny * P.gy * wz + nz * P.gz * wy;
  wby += nx * P.gx * wz + nz * P.gz * wx;
  wbz += nx * P.gx * wy + ny * P.gy * wx;
  yb[WX] += wbx; yb[WX + 1] += wby; yb[WX + 2] += wbz;
  // rotors: s_i = Omega_i^2 through the thrust and torque rows of G
  const float a0 = P.T2c * T2b, a1 = P.txc * nx, a2 = P.tyc * ny, a3 = P.tzc * nz;
  Omb[0] = 2.f * Om[0] * ((a0 + a1) + (a3 - a2));
  Omb[1] = 2.f * Om[1] * ((a0 - a1) - (a2 + a3));
  Omb[2] = 2.f * Om[2] * ((a0 - a1) + (a2 + a3));
  Omb[3] = 2.f * Om[3] * ((a0 + a1) + (a2 - a3));
}

// Adds the m and J cotangents that the derived constants' cotangents dc
// carry: T2c = 2 kt / m and cd_m = c_d / m (d/dm = -T2c / m, -cd_m / m);
// gx = (Jy - Jz) / Jx, gy = (Jz - Jx) / Jy, gz = (Jx - Jy) / Jz, txc ~ 1 / Jx,
// tyc ~ 1 / Jy, tzc ~ 1 / Jz.
__device__ __forceinline__ void theta_from_derived(const DevGroup& P, const float dc[NDC], float tb[NTH]) {
  tb[TH_M] -= (dc[DC_T2] * P.T2c + dc[DC_CD] * P.cd_m) * P.inv_m;
  tb[TH_J] += dc[DC_GZ] * P.iJz - dc[DC_GY] * P.iJy - (dc[DC_GX] * P.gx + dc[DC_TX] * P.txc) * P.iJx;
  tb[TH_J + 1] += dc[DC_GX] * P.iJx - dc[DC_GZ] * P.iJz - (dc[DC_GY] * P.gy + dc[DC_TY] * P.tyc) * P.iJy;
  tb[TH_J + 2] += dc[DC_GY] * P.iJy - dc[DC_GX] * P.iJx - (dc[DC_GZ] * P.gz + dc[DC_TZ] * P.tzc) * P.iJz;
}

// Cotangent of the controller: ub (rotor commands) -> xb (state), tb (theta).
// PID: also eb, the cotangent of the rate error e the integrator consumed;
// adds the integral term's share to xb[XI..] and writes wdb, the cotangent of
// omega' (wdot, at x), for the caller to carry through Eq. (qd4).
// C: the controller's values at x (controller_fwd).
template <bool PID = false>
__device__ __forceinline__ void controller_vjp(const DevGroup& P, const float* x, const Hd& hd, const Ctl& C,
                                               const float ub[4], float* xb, float tb[NTH],
                                               const float* eb = nullptr, float* wdb = nullptr) {
  // u = omega_max sqrt(clamp(S, 0, 1)) (S in units of omega_max^2): gradient
  // passes on 0 < S <= 1 (sqrt'(0) taken as 0)
  float Sb[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float s = C.S[i];
    Sb[i] = (s > 0.f && s <= 1.f) ? ub[i] * (0.5f * P.omax) * rsqrtf(s) : 0.f;
  }
  const float f0b = (Sb[0] + Sb[1]) + (Sb[2] + Sb[3]);
  float fb[3];
  fb[0] = (Sb[0] - Sb[1]) + (Sb[3] - Sb[2]);
  fb[1] = (Sb[2] + Sb[3]) - (Sb[0] + Sb[1]);
  fb[2] = (Sb[0] - Sb[1]) + (Sb[2] - Sb[3]);
  // f_i = mt_i krate_i (2 katt_i qe_i - omega_i); qe = s E, s = sign(E_w) / |Q|
  float Eb[4], kap = 0.f;
  Eb[0] = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    tb[TH_KRATE + i] += fb[i] * P.mt[i] * (P.katt2[i] * C.qe[1 + i] - x[WX + i]);
    tb[TH_KATT + i] += fb[i] * P.wa[i] * 2.f * C.qe[1 + i];
    xb[WX + i] -= fb[i] * P.wa[i];
    float qeb = fb[i] * P.qa[i];
    if (PID) {
      // e_i = 2 katt_i qe_i - omega_i feeds the integrator; f_i also holds
      // mix_i taumax_i (kI_i xi_i - kD_i omega'_i)
      qeb += eb[i] * P.katt2[i];
      tb[TH_KATT + i] += eb[i] * 2.f * C.qe[1 + i];
      xb[WX + i] -= eb[i];
      xb[XI + i] += fb[i] * P.kic[i];
      wdb[i] = -fb[i] * P.kdc[i];
    }
    kap += qeb * C.qe[1 + i];
    Eb[1 + i] = qeb * C.s;
  }
  // E = conj(q) o Q
  const float w = x[QW], qx = x[QX], qy = x[QY], qz = x[QZ];
  const float dw = C.Q[0], dx = C.Q[1], dy = C.Q[2], dz = C.Q[3];
  const float Ew = Eb[0], Ex = Eb[1], Ey = Eb[2], Ez = Eb[3];
  float qbw = Ew * dw + Ex * dx + Ey * dy + Ez * dz;
  float qbx = Ew * dx - Ex * dw + Ey * dz - Ez * dy;
  float qby = Ew * dy - Ex * dz - Ey * dw + Ez * dx;
  float qbz = Ew * dz + Ex * dy - Ey * dx - Ez * dw;
  // |Q|^-1 enters qe: d(1/|Q|)/dQ = -Q / |Q|^3
  const float G = -kap * C.s * C.s;
  float Qb[4];
  Qb[0] = Ew * w - Ex * qx - Ey * qy - Ez * qz + G * dw;
  Qb[1] = Ew * qx + Ex * w - Ey * qz + Ez * qy + G * dx;
  Qb[2] = Ew * qy + Ex * qz + Ey * w - Ez * qx + G * dy;
  Qb[3] = Ew * qz - Ex * qy + Ey * qx + Ez * w + G * dz;
  // Q = q_z(psi) o (X0 Y0, X1 Y0, X0 Y1, X1 Y1)
  const float P0b = hd.c2 * Qb[0] + hd.s2 * Qb[3];
  const float P1b = hd.c2 * Qb[1] + hd.s2 * Qb[2];
  const float P2b = hd.c2 * Qb[2] - hd.s2 * Qb[1];
  const float P3b = hd.c2 * Qb[3] - hd.s2 * Qb[0];
  const float X0b = P0b * C.Y[0] + P2b * C.Y[1], X1b = P1b * C.Y[0] + P3b * C.Y[1];
  const float Y0b = P0b * C.X[0] + P1b * C.X[1], Y1b = P2b * C.X[0] + P3b * C.X[1];
  // Y = (M + N, A); X = (N + F_z, -B) or (-B, N - F_z)
  float Nb = Y0b, Ab = Y1b, Bb, Fzb;
  if (C.up) { Nb += X0b; Fzb = X0b; Bb = -X1b; }
  else { Nb += X1b; Fzb = -X1b; Bb = -X0b; }
  // M = sqrt(A^2 + N^2), N = sqrt(B^2 + F_z^2)
  const float M2b = 0.5f * Y0b * C.rM;
  Ab += 2.f * C.A * M2b;
  const float N2b = M2b + 0.5f * Nb * C.rN;
  Bb += 2.f * C.B * N2b;
  Fzb += 2.f * C.F[2] * N2b;
  // (A, B) = heading rotation of (F_x, F_y); f0 = f0c (F . b3) / 2, f0c = m / (2 kt omega_max^2)
  const float fcb = 0.5f * f0b * P.f0c;
  tb[TH_M] += f0b * C.fc * P.mix0;
  float Fb[3];
  Fb[0] = hd.c * Ab - hd.s * Bb + fcb * C.b3[0];
  Fb[1] = hd.s * Ab + hd.c * Bb + fcb * C.b3[1];
  Fb[2] = Fzb + fcb * C.b3[2];
  // b3 = R(q) e3 -> q
  const float bbx = fcb * C.F[0], bby = fcb * C.F[1], bbz = fcb * C.F[2];
  qbw += 2.f * (qy * bbx - qx * bby);
  qbx += 2.f * (qz * bbx - w * bby) - 4.f * qx * bbz;
  qby += 2.f * (w * bbx + qz * bby) - 4.f * qy * bbz;
  qbz += 2.f * (qx * bbx + qy * bby);
  xb[QW] += qbw; xb[QX] += qbx; xb[QY] += qby; xb[QZ] += qbz;
  // F = a + g e3, a = clamp(kp e - kd v)
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float arb = C.pass[i] ? Fb[i] : 0.f;
    tb[TH_KP + i] += arb * C.e[i];
    tb[TH_KD + i] -= arb * x[VX + i];
    xb[PX + i] -= P.kp[i] * arb;
    xb[VX + i] -= P.kd[i] * arb;
  }
}

// Adjoint of one RK4 step x_n -> x_{n+1}: lam <- (d x_{n+1} / d x_n)^T lam,
// tb += (d x_{n+1} / d theta)^T lam (the controller's gains and m), dc += the
// derived constants' share (theta_from_derived).  x is the step-start state.
// The controller is evaluated twice: for the rotor commands the stages need,
// and again for the values its VJP needs at the end (keeping them from the
// first evaluation, in registers or in a shared-memory stash, measured
// slower: the recomputation fills issue slots that would otherwise wait).
template <int MODE>
__device__ __forceinline__ void step_vjp(const DevGroup& P, const St& x, const float4 c, const Hd& hd,
                                         const StepH& H, const LinCoef& L, St& lam, float tb[NTH], float dc[NDC]) {
  float dOm[4], bq[3];
  float wdot[3], e[3];  // PID: omega' at x and the rate error
  thrust_axis(x.a + QW, bq);
  if (MODE == 0) {
    dOm[0] = c.x - x.a[OM]; dOm[1] = c.y - x.a[OM + 1]; dOm[2] = c.z - x.a[OM + 2]; dOm[3] = c.w - x.a[OM + 3];
  } else {
    float r[4];
    if (MODE == 2) {
      // omega' at x (the first RK4 stage's) feeds the derivative term
      float k0[NRB];
      rb_derivative(P, x.a, x.a + OM, k0);
      wdot[0] = k0[WX]; wdot[1] = k0[WX + 1]; wdot[2] = k0[WX + 2];
      Ctl C;
      controller_fwd<true>(P, x.a, c, hd, bq, C, r, wdot, e);
    } else {
      controller(P, x.a, c, hd, bq, r);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) dOm[i] = fmaf(P.omax, r[i], -x.a[OM + i]);  // u = omega_max r
  }
  // rotor lag: stage k sees Omega + c_k (u - Omega) (c_1 = 0); the step ends
  // at Omega + c5 (u - Omega).  Stage rotor speeds are recomputed where used
  // and each stage's cotangent is folded into ub / xb at once.
  float Om[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) Om[i] = x.a[OM + i] + L.c2 * dOm[i];
  float k[NRB], y2[NRB], y3[NRB], y4[NRB];
  rb_derivative(P, x.a, x.a + OM, k);
#pragma unroll
  for (int i = 0; i < NRB; ++i) y2[i] = x.a[i] + coef(i, H.h2, H.h2q) * k[i];
  rb_derivative(P, y2, Om, k);
#pragma unroll
  for (int i = 0; i < 4; ++i) Om[i] = x.a[OM + i] + L.c3 * dOm[i];
#pragma unroll
  for (int i = 0; i < NRB; ++i) y3[i] = x.a[i] + coef(i, H.h2, H.h2q) * k[i];
  rb_derivative(P, y3, Om, k);
#pragma unroll
  for (int i = 0; i < 4; ++i) Om[i] = x.a[OM + i] + L.c4 * dOm[i];
#pragma unroll
  for (int i = 0; i < NRB; ++i) y4[i] = x.a[i] + coef(i, H.h, H.hq) * k[i];
  float xb[NXP], g[NRB], yb[NRB], Ob[4], ub[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ub[i] = L.c5 * lam.a[OM + i];
    xb[OM + i] = lam.a[OM + i] - ub[i];
  }
#pragma unroll
  for (int i = 0; i < NRB; ++i) { xb[i] = lam.a[i]; g[i] = coef(i, H.h6, H.h6q) * lam.a[i]; yb[i] = 0.f; }
  rb_derivative_vjp(P, y4, Om, g, yb, Ob, dc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ub[i] += L.c4 * Ob[i];
    xb[OM + i] += Ob[i] - L.c4 * Ob[i];
    Om[i] = x.a[OM + i] + L.c3 * dOm[i];
  }
#pragma unroll
  for (int i = 0; i < NRB; ++i) {
    xb[i] += yb[i];
    g[i] = 2.f * coef(i, H.h6, H.h6q) * lam.a[i] + coef(i, H.h, H.hq) * yb[i];
    yb[i] = 0.f;
  }
  rb_derivative_vjp(P, y3, Om, g, yb, Ob, dc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ub[i] += L.c3 * Ob[i];
    xb[OM + i] += Ob[i] - L.c3 * Ob[i];
    Om[i] = x.a[OM + i] + L.c2 * dOm[i];
  }
#pragma unroll
  for (int i = 0; i < NRB; ++i) {
    xb[i] += yb[i];
    g[i] = 2.f * coef(i, H.h6, H.h6q) * lam.a[i] + coef(i, H.h2, H.h2q) * yb[i];
    yb[i] = 0.f;
  }
  rb_derivative_vjp(P, y2, Om, g, yb, Ob, dc);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ub[i] += L.c2 * Ob[i];
    xb[OM + i] += Ob[i] - L.c2 * Ob[i];
  }
#pragma unroll
  for (int i = 0; i < NRB; ++i) {
    xb[i] += yb[i];
    g[i] = coef(i, H.h6, H.h6q) * lam.a[i] + coef(i, H.h2, H.h2q) * yb[i];
    yb[i] = 0.f;
  }
  rb_derivative_vjp(P, x.a, x.a + OM, g, yb, Ob, dc);
#pragma unroll
  for (int i = 0; i < 4; ++i) xb[OM + i] += Ob[i];
#pragma unroll
  for (int i = 0; i < NRB; ++i) xb[i] += yb[i];
  if (MODE == 2) {
    // xi' = clamp(xi + h e): the gradient passes where the clamp does not bind
    float eb[3], wdb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float v = x.a[XI + i] + H.h * e[i];
      const bool pass = (v >= -P.xim[i]) && (v <= P.xim[i]);
      xb[XI + i] = pass ? lam.a[XI + i] : 0.f;
      eb[i] = pass ? H.h * lam.a[XI + i] : 0.f;
    }
    Ctl C;
    float r2[4], e2[3];
    controller_fwd<true>(P, x.a, c, hd, bq, C, r2, wdot, e2);
    controller_vjp<true>(P, x.a, hd, C, ub, xb, tb, eb, wdb);
    // omega' = rows WX.. of Eq. (qd4) at (x, Omega)
#pragma unroll
    for (int i = 0; i < NRB; ++i) { g[i] = 0.f; yb[i] = 0.f; }
    g[WX] = wdb[0]; g[WX + 1] = wdb[1]; g[WX + 2] = wdb[2];
    rb_derivative_vjp(P, x.a, x.a + OM, g, yb, Ob, dc);
#pragma unroll
    for (int i = 0; i < NRB; ++i) xb[i] += yb[i];
#pragma unroll
    for (int i = 0; i < 4; ++i) xb[OM + i] += Ob[i];
  } else if (MODE == 1) {
    Ctl C;
    float r2[4];
    controller_fwd(P, x.a, c, hd, bq, C, r2);
    controller_vjp(P, x.a, hd, C, ub, xb, tb);
  }
#pragma unroll
  for (int i = 0; i < state_dim<MODE>(); ++i) lam.a[i] = xb[i];
}

}  // namespace qs
