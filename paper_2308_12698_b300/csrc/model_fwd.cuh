// Device model of one quadrotor step, one thread per agent, FP32 in registers.
//
//   rb_derivative   Eq. (qd1)-(qd4), Eq. (2), Eq. (3) of arXiv 2308.12698 Sec. III-B,
//                   plus linear drag, for the 13 rigid-body components
//   rotor lag       Omega' = (Omega_cmd - Omega)/tau_m; linear and decoupled, so
//                   its four RK4 stages and the RK4 update are applied through
//                   their exact coefficients (LinCoef) instead of four
//                   derivative evaluations -- the same RK4 map, fewer operations
//   drag            linear in v with a forcing that does not depend on v: the
//                   translation's RK4 update is likewise a fixed weighting of
//                   v and the four stages' thrust S b (LinCoef, whose weights
//                   also carry the thrust constant and gravity)
//   controller      cascaded position PD -> attitude P -> normalised rate P ->
//                   G^-1 -> rotor clamp, the mixer in units of omega_max^2 so
//                   that the clamp is a saturating add (the paper's inner body-rate loop,
//                   Sec. III-B, completed as documented in quadsim.h).  The
//                   desired attitude (body z along the demanded force, body y
//                   normal to it and to the heading) is the rotation
//                   Rz(psi) Rx(phi) Ry(theta); its quaternion is formed from
//                   unnormalised half-angle pairs and normalised once -- the
//                   same rotation as building the matrix and converting it
//                   (Shepperd), without the matrix or the branch
//   PID rate loop   MODE 2 (the paper's "PID body rate controller", Sec. III-B):
//                   adds taumax (kI xi - kD omega') to the rate loop's torque,
//                   omega' on the measurement (Eq. qd4 at the step start, the
//                   first RK4 stage's derivative), xi <- clamp(xi + h e) once
//                   per step
//   rk4             classical RK4, command held over the stages (Sec. III-B)
//   (the vector-Jacobian products of the adjoint are in model_adj.cuh)
//
// State index map (17 floats): p 0-2, v 3-5, q 6-9 (w x y z), omega 10-12,
// Omega 13-16; in the PID mode (MODE 2) also xi 17-19, the integral of the
// body-rate error.  rb_derivative returns 2 q' for the quaternion
// (q o [0, w]), and the RK4 coefficients of those four components are halved
// to match.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "checks.cuh"

namespace qs {

enum { PX = 0, VX = 3, QW = 6, QX = 7, QY = 8, QZ = 9, WX = 10, OM = 13, NX = 17, NRB = 13, XI = 17, NXP = 20 };
enum { TH_KP = 0, TH_KD = 3, TH_KATT = 6, TH_KRATE = 9, TH_M = 12, TH_J = 13, NTH = 16 };

// Per-group constants, derived on the host in double from the public
// parameters and rounded once to float.  Rows of four floats.
struct __align__(16) DevGroup {
  // forward: dynamics
  float T2c, cd_m, g, inv_tau;  // 2 kt / m, c_d / m, gravity, 1 / tau_m
  float txc, tyc, tzc, omax;    // kt L sin(a) / Jx, kt L cos(a) / Jy, kq / Jz, omega_max
  float gx, gy, gz, m;          // (Jy - Jz)/Jx, (Jz - Jx)/Jy, (Jx - Jy)/Jz, mass
  // forward: controller.  The mixer works in units of omega_max^2 (its
  // constants below are divided by omega_max^2), so the rotor clamp
  // [0, omega_max^2] is a saturation to [0, 1].
  float kp[3], a_max;
  float kd[3], f0c;             // f0c = m / (2 kt omega_max^2): F . R(q) e3 / 2 -> Omega^2 per rotor
  float qa[3], az_lo;           // mix_i krate_i taumax_i 2 katt_i: error-quaternion component -> Omega^2; g - a_max
  float wa[3], az_hi;           // mix_i krate_i taumax_i: body rate -> Omega^2; g + a_max
  // adjoint
  float inv_m, Jx, Jy, Jz;
  float iJx, iJy, iJz, mix0;    // mix0 = 1 / (4 kt omega_max^2)
  float krate[3], gxt;          // gxt, gyt, gzt: the gyroscopic coefficients over the torque ones,
  float katt2[3], gyt;          // (Jy - Jz) / (kt L sin a), (Jz - Jx) / (kt L cos a), (Jx - Jy) / kq
  float mt[3], gzt;             // mix_i taumax_i  (mix = 1/(4 kt L sin a), 1/(4 kt L cos a), 1/(4 kq))
  // forward: PID rate loop (MODE 2)
  float kic[3], pad5;           // mix_i taumax_i kI_i: rate-error integral -> Omega^2
  float kdc[3], pad6;           // mix_i taumax_i kD_i: angular acceleration -> Omega^2
  float xim[3], pad7;           // integrator limit |xi_i| <= xim_i
  // agent type (0 quadrotor, 1 car, 2 fixed-wing) and the vehicle model's constants:
  // car (tan(delta_max)/L_w, a_max, k_v, l_min), fixed-wing (b_phi, phi_max, k_chi, b_hd, b_h, b_V)
  float vt, vk[6], pad8;
};
static_assert(sizeof(DevGroup) == 68 * 4, "DevGroup layout");

// Components of an agent's state in a mode: 17, or 20 with the PID integral.
template <int MODE>
__host__ __device__ constexpr int state_dim() {
  return MODE == 2 ? NXP : NX;
}

struct St {
  float a[NXP];  // the first state_dim<MODE>() are used
};

// Commanded heading psi: cos, sin of psi and of psi / 2.
struct Hd {
  float c, s, c2, s2;
};

__device__ __forceinline__ Hd heading(float psi) {
  Hd h;
  sincosf(psi, &h.s, &h.c);
  sincosf(0.5f * psi, &h.s2, &h.c2);
  return h;
}

// Step-size constants rounded once on the host.  q components use halved
// coefficients because rb_derivative returns 2 q'.
struct StepH {
  float h, h2, h6;      // h, h/2, h/6
  float hq, h2q, h6q;   // h/2, h/4, h/12
};

__device__ __forceinline__ float coef(int i, float a, float aq) { return (i >= QW && i <= QZ) ? aq : a; }

// Correctly rounded FP32 operations, one rounding each, the same on the host
// and the device (the device would otherwise contract a * b + c into an FMA):
// coefficients computed with them agree bit for bit wherever they are made.
__host__ __device__ __forceinline__ float rmul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float radd(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float rsub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}

// Exact RK4 weights of the step's linear parts, per group and step size.
// Rotor lag Omega' = (u - Omega)/tau: stage k sees Omega + c_k (u - Omega)
// (c_1 = 0), and the step ends at Omega + c5 (u - Omega).
// Drag: v' = T2c f_k - g e3 - a v with a = c_d / m and f_k = S_k b_k the
// stage's thrust (rb_stage), which does not depend on v, so RK4's stage
// velocities and sums reduce to
//   v_new = v + (am1 v + B1 f1 + B2 f2 + B3 f3 + B4 f4 + gb e3)
//   p_new = p + (g v + D1 f1 + D2 f2 + D3 f3 + gd e3)
// with B_k = T2c b_k, D_k = T2c d_k, gb = -g (b1 + b2 + b3 + b4),
// gd = -g (d1 + d2 + d3) and, for z = a h,
//   am1 = -z + z^2/2 - z^3/6 + z^4/24   (RK4's e^-z - 1)
//   b = h/6 (1 - z + z^2/2 - z^3/4, 2 - z + z^2/2, 2 - z, 1)
//   g = h/6 (6 - 3z + z^2 - z^3/4),  d = h^2/6 (1 - z/2 + z^2/4, 1 - z/2, 1)
// the same map as the four stages, in fewer operations.  One-group launches
// take them from the kernel's parameters (computed on the host), so that the
// step's multiply-adds read them from the constant bank, not registers.
struct LinCoef {
  float c2, c3, c4, c5;
  float am1, b1, b2, b3, b4;  // B_k: times T2c
  float g, d1, d2, d3;        // D_k: times T2c
  float gb, gd;               // gravity's share of the v and p updates (z only)
  float t2[3], t1[3], t6[3];  // h/2, h, h/6 times the torque coefficients txc, tyc, tzc
};

__host__ __device__ __forceinline__ LinCoef lin_coef(const DevGroup& P, const StepH& H) {
  LinCoef L;
  L.c2 = rmul(H.h2, P.inv_tau);
  L.c3 = rmul(L.c2, rsub(1.f, L.c2));
  L.c4 = rmul(rmul(H.h, P.inv_tau), rsub(1.f, L.c3));
  L.c5 = rmul(rmul(H.h6, P.inv_tau), radd(rsub(3.f, rmul(2.f, L.c2)), rsub(rsub(3.f, rmul(2.f, L.c3)), L.c4)));
  const float z = rmul(H.h, P.cd_m);
  L.am1 = rmul(-z, rsub(1.f, rmul(z, rsub(0.5f, rmul(z, rsub(1.f / 6.f, rmul(z, 1.f / 24.f)))))));
  const float b1 = rmul(H.h6, rsub(1.f, rmul(z, rsub(1.f, rmul(z, rsub(0.5f, rmul(z, 0.25f)))))));
  const float b2 = rmul(H.h6, rsub(2.f, rmul(z, rsub(1.f, rmul(z, 0.5f)))));
  const float b3 = rmul(H.h6, rsub(2.f, z));
  const float b4 = H.h6;
  L.g = rmul(H.h6, rsub(6.f, rmul(z, rsub(3.f, rmul(z, rsub(1.f, rmul(z, 0.25f)))))));
  const float hh6 = rmul(H.h, H.h6);
  const float d1 = rmul(hh6, rsub(1.f, rmul(z, rsub(0.5f, rmul(z, 0.25f)))));
  const float d2 = rmul(hh6, rsub(1.f, rmul(z, 0.5f)));
  const float d3 = hh6;
  L.b1 = rmul(P.T2c, b1); L.b2 = rmul(P.T2c, b2); L.b3 = rmul(P.T2c, b3); L.b4 = rmul(P.T2c, b4);
  L.d1 = rmul(P.T2c, d1); L.d2 = rmul(P.T2c, d2); L.d3 = rmul(P.T2c, d3);
  L.gb = rmul(-P.g, radd(radd(radd(b1, b2), b3), b4));
  L.gd = rmul(-P.g, radd(radd(d1, d2), d3));
  const float tc[3] = {P.txc, P.tyc, P.tzc};
  for (int i = 0; i < 3; ++i) {
    L.t2[i] = rmul(H.h2, tc[i]);
    L.t1[i] = rmul(H.h, tc[i]);
    L.t6[i] = rmul(H.h6, tc[i]);
  }
  return L;
}

// ------------------------------------------------------------ planar I/O --
// Plane k (0..3) holds float4 of components 4k..4k+3; plane 4 holds
// component 16 (a float per agent), or components 16..19 (a float4 per
// agent) when the state has 20 components.
template <int NS = NX>
__device__ __forceinline__ void load_state(const float* __restrict__ base, int64_t n, int64_t i, St& x) {
#ifdef QS_CHECKED
  if (!QS_OK(i >= 0 && i < n, 1, i)) {
    for (int k = 0; k < NS; ++k) x.a[k] = 0.f;
    return;
  }
#endif
  const float4* P = reinterpret_cast<const float4*>(base);
  const float4 a = P[i], b = P[n + i], c = P[2 * n + i], d = P[3 * n + i];
  x.a[0] = a.x; x.a[1] = a.y; x.a[2] = a.z; x.a[3] = a.w;
  x.a[4] = b.x; x.a[5] = b.y; x.a[6] = b.z; x.a[7] = b.w;
  x.a[8] = c.x; x.a[9] = c.y; x.a[10] = c.z; x.a[11] = c.w;
  x.a[12] = d.x; x.a[13] = d.y; x.a[14] = d.z; x.a[15] = d.w;
  if (NS == NXP) {
    const float4 e = P[4 * n + i];
    x.a[16] = e.x; x.a[17] = e.y; x.a[18] = e.z; x.a[19] = e.w;
  } else {
    x.a[16] = base[16 * n + i];
  }
}

template <int NS = NX>
__device__ __forceinline__ void store_state(float* __restrict__ base, int64_t n, int64_t i, const St& x) {
#ifdef QS_CHECKED
  if (!QS_OK(i >= 0 && i < n, 2, i)) return;
#endif
  float4* P = reinterpret_cast<float4*>(base);
  P[i] = make_float4(x.a[0], x.a[1], x.a[2], x.a[3]);
  P[n + i] = make_float4(x.a[4], x.a[5], x.a[6], x.a[7]);
  P[2 * n + i] = make_float4(x.a[8], x.a[9], x.a[10], x.a[11]);
  P[3 * n + i] = make_float4(x.a[12], x.a[13], x.a[14], x.a[15]);
  if (NS == NXP)
    P[4 * n + i] = make_float4(x.a[16], x.a[17], x.a[18], x.a[19]);
  else
    base[16 * n + i] = x.a[16];
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// The SFU's approximate reciprocal square root and square root, subnormal
// inputs flushed to zero (PTX rsqrt.approx.ftz.f32, sqrt.approx.ftz.f32): one
// instruction each.  The controller's arguments are squared norms of order g^2
// or a clamped rotor demand in [0, Omega_max^2], never subnormal where it
// matters.  Against the rsqrtf / s * rsqrtf(s) forms (which also handle
// subnormals) the fused step ran 6.5 % faster, within the same parity bars.
__device__ __forceinline__ float rsqrt_sfu(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float sqrt_sfu(float v) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// ---------------------------------------------------- rigid-body derivative --
// y: the 13 rigid-body components at a stage; Om: the stage's rotor speeds.
// d[0..2] = v, d[3..5] = v', d[6..9] = 2 q', d[10..12] = omega'.
__device__ __forceinline__ void rb_derivative(const DevGroup& P, const float* y, const float Om[4], float* d) {
  const float s1 = Om[0] * Om[0], s2 = Om[1] * Om[1], s3 = Om[2] * Om[2], s4 = Om[3] * Om[3];
  // Eq. (2)-(3): collective thrust (as 2 f_c / m) and body torques (as tau / J)
  const float T2 = P.T2c * ((s1 + s2) + (s3 + s4));
  const float tx = P.txc * ((s1 - s2) + (s4 - s3));
  const float ty = P.tyc * ((s3 + s4) - (s1 + s2));
  const float tz = P.tzc * ((s1 - s2) + (s3 - s4));
  const float w = y[QW], qx = y[QX], qy = y[QY], qz = y[QZ];
  const float wx = y[WX], wy = y[WX + 1], wz = y[WX + 2];
  // R(q) e3 = (2 bx, 2 by, 1 - 2 bxy)
  const float bx = qx * qz + w * qy, by = qy * qz - w * qx, bxy = qx * qx + qy * qy;
  // Eq. (qd1)
  d[0] = y[VX]; d[1] = y[VX + 1]; d[2] = y[VX + 2];
  // Eq. (qd2) with linear drag
  d[3] = T2 * bx - P.cd_m * y[VX];
  d[4] = T2 * by - P.cd_m * y[VX + 1];
  d[5] = (0.5f * T2 - P.g) - T2 * bxy - P.cd_m * y[VX + 2];
  // Eq. (qd3), doubled: q o [0, omega]
  d[QW] = -qx * wx - qy * wy - qz * wz;
  d[QX] = w * wx + qy * wz - qz * wy;
  d[QY] = w * wy + qz * wx - qx * wz;
  d[QZ] = w * wz + qx * wy - qy * wx;
  // Eq. (qd4): omega' = I^-1 (tau - omega x I omega), diagonal I
  d[WX] = P.gx * (wy * wz) + tx;
  d[WX + 1] = P.gy * (wz * wx) + ty;
  d[WX + 2] = P.gz * (wx * wy) + tz;
}

// Half the body z axis, b = R(q) e3 / 2 = (qx qz + w qy, qy qz - w qx,
// 1/2 - qx^2 - qy^2): the thrust direction of Eq. (qd2), at each RK4 stage and
// in the controller at the step start (the same bits: the step shares them).
__device__ __forceinline__ void thrust_axis(const float q[4], float b[3]) {
  b[0] = fmaf(q[1], q[3], __fmul_rn(q[0], q[2]));
  b[1] = fmaf(q[2], q[3], -__fmul_rn(q[0], q[1]));
  b[2] = fmaf(-q[1], q[1], fmaf(-q[2], q[2], 0.5f));
}

// The same derivative at an RK4 stage, for the forward step: the rotation's
// components, 2 q' and omega' over the torque coefficients (dw_i = omega'_i /
// t_i with t = (txc, tyc, tzc): the gyroscopic term's coefficient divided by
// t_i, and t_i carried by the RK4 weights of omega, lin_coef's t2, t1, t6:
// three multiplies fewer per stage), and the thrust as f = S b with S the sum
// of the Omega_i^2 and b = thrust_axis(q) (also returned): v' = T2c f - g e3 -
// cd_m v, whose constants lin_coef's weights carry.
// Wherever two products meet one sum the multiply-add is written out (fmaf,
// __fmul_rn), so that each kernel that steps agents computes the same bits: the
// checkpoints of one kernel and the states another recomputes from them must
// agree, and a compiler free to fuse either product could round differently
// in different kernels.
__device__ __forceinline__ void rb_stage(const DevGroup& P, const float q[4], const float w[3], const float Om[4],
                                         float f[3], float dq[4], float dw[3], float b[3]) {
  // s_i = Omega_i^2 enter only as sums and differences of pairs, each one
  // multiply-add: s1 +- s2 = fma(Om1, Om1, +-s2), s3 +- s4 likewise
  const float s2 = __fmul_rn(Om[1], Om[1]), s4 = __fmul_rn(Om[3], Om[3]);
  const float s12 = fmaf(Om[0], Om[0], s2), d12 = fmaf(Om[0], Om[0], -s2);
  const float s34 = fmaf(Om[2], Om[2], s4), d34 = fmaf(Om[2], Om[2], -s4);
  const float S = __fadd_rn(s12, s34);
  // Eq. 3's torque rows without their coefficients
  const float tx = __fsub_rn(d12, d34), ty = __fsub_rn(s34, s12), tz = __fadd_rn(d12, d34);
  thrust_axis(q, b);
  f[0] = __fmul_rn(S, b[0]);
  f[1] = __fmul_rn(S, b[1]);
  f[2] = __fmul_rn(S, b[2]);
  dq[0] = fmaf(-q[3], w[2], fmaf(-q[2], w[1], -__fmul_rn(q[1], w[0])));
  dq[1] = fmaf(-q[3], w[1], fmaf(q[2], w[2], __fmul_rn(q[0], w[0])));
  dq[2] = fmaf(-q[1], w[2], fmaf(q[3], w[0], __fmul_rn(q[0], w[1])));
  dq[3] = fmaf(-q[2], w[0], fmaf(q[1], w[1], __fmul_rn(q[0], w[2])));
  dw[0] = fmaf(P.gxt, __fmul_rn(w[1], w[2]), tx);
  dw[1] = fmaf(P.gyt, __fmul_rn(w[2], w[0]), ty);
  dw[2] = fmaf(P.gzt, __fmul_rn(w[0], w[1]), tz);
}

// a + b and a - b saturated to [0, 1], NaN to 0 (PTX add.sat / sub.sat): the
// mixer's last add and the rotor clamp in one instruction.
__device__ __forceinline__ float add_sat(float a, float b) {
  float r;
  asm("add.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float sub_sat(float a, float b) {
  float r;
  asm("sub.rn.sat.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// ---------------------------------------------------------- the controller --
struct Ctl {
  float e[3];
  bool pass[3];  // acceleration clamp passes the gradient
  float F[3];    // desired acceleration plus gravity (the desired force / m)
  float b3[3], fc;
  float A, B;    // F in the heading frame: along and across (cos psi, sin psi, 0)
  float N, rN;   // |(B, F_z)| and its reciprocal
  float M, rM;   // |F| and its reciprocal
  bool up;       // F_z >= 0: which half-angle formula of the roll
  float X[2];    // roll half-angle (cos, sin), unnormalised
  float Y[2];    // pitch half-angle (cos, sin), unnormalised
  float Q[4];    // q_d unnormalised
  float E[4];    // conj(q) o Q
  float s;       // sign(E_w) / |Q|
  float qe[4];
  float S[4];    // Omega^2 / omega_max^2 demanded by the mixer, before the clamp
};

// b: thrust_axis(q) at x (the first RK4 stage's).  r receives the rotor
// commands as fractions of omega_max, sqrt(clamp(S, 0, 1)).
// PID: also the integral and derivative terms of the rate loop (x holds xi at
// XI..XI+2, wdot is omega' at x); e receives the rate error omega_des - omega.
template <bool PID = false>
__device__ __forceinline__ void controller_fwd(const DevGroup& P, const float* x, const float4 c, const Hd& hd,
                                               const float b[3], Ctl& C, float r[4], const float* wdot = nullptr,
                                               float* e = nullptr) {
  const float cc[3] = {c.x, c.y, c.z};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    C.e[i] = cc[i] - x[PX + i];
    const float ar = P.kp[i] * C.e[i] - P.kd[i] * x[VX + i];
    C.pass[i] = (ar >= -P.a_max) && (ar <= P.a_max);
    C.F[i] = clampf(ar, -P.a_max, P.a_max);
  }
  // z: gravity added before the clamp, whose bounds are then g -+ a_max
  C.e[2] = cc[2] - x[PX + 2];
  const float az = fmaf(P.kp[2], C.e[2], fmaf(-P.kd[2], x[VX + 2], P.g));
  C.pass[2] = (az >= P.az_lo) && (az <= P.az_hi);
  C.F[2] = clampf(az, P.az_lo, P.az_hi);
  const float w = x[QW], qx = x[QX], qy = x[QY], qz = x[QZ];
  // collective thrust demand F . R(q) e3 = 2 (F . b)
  C.b3[0] = 2.f * b[0];
  C.b3[1] = 2.f * b[1];
  C.b3[2] = 2.f * b[2];
  const float fh = fmaf(C.F[0], b[0], fmaf(C.F[1], b[1], __fmul_rn(C.F[2], b[2])));
  C.fc = 2.f * fh;
  // R_des = Rz(psi) Rx(phi) Ry(theta): in the heading frame the desired z axis is
  // (A, B, F_z) / |F| = (sin theta, -sin phi cos theta, cos phi cos theta)
  C.A = hd.c * C.F[0] + hd.s * C.F[1];
  C.B = hd.c * C.F[1] - hd.s * C.F[0];
  const float N2 = C.B * C.B + C.F[2] * C.F[2];
  C.rN = rsqrt_sfu(N2);
  C.N = N2 * C.rN;
  const float M2 = C.A * C.A + N2;
  C.rM = rsqrt_sfu(M2);
  C.M = M2 * C.rM;
  // half angles as unnormalised (cos, sin) pairs: (N + F_z, -B) ~ (1 + cos phi, sin phi),
  // or (-B, N - F_z) ~ (sin phi, 1 - cos phi) when F_z < 0 (both N + |F_z|); (M + N, A) for theta
  C.up = C.F[2] >= 0.f;
  const float Xa = C.N + fabsf(C.F[2]);
  C.X[0] = C.up ? Xa : -C.B;
  C.X[1] = C.up ? -C.B : Xa;
  C.Y[0] = C.M + C.N;
  C.Y[1] = C.A;
  // q_d ~ q_z(psi) o q_x(phi) o q_y(theta)
  const float P0 = C.X[0] * C.Y[0], P1 = C.X[1] * C.Y[0], P2 = C.X[0] * C.Y[1], P3 = C.X[1] * C.Y[1];
  C.Q[0] = hd.c2 * P0 - hd.s2 * P3;
  C.Q[1] = hd.c2 * P1 - hd.s2 * P2;
  C.Q[2] = hd.c2 * P2 + hd.s2 * P1;
  C.Q[3] = hd.c2 * P3 + hd.s2 * P0;
  // q_e = conj(q) o q_d, shortest way round
  const float dw = C.Q[0], dx = C.Q[1], dy = C.Q[2], dz = C.Q[3];
  C.E[0] = w * dw + qx * dx + qy * dy + qz * dz;
  C.E[1] = w * dx - dw * qx - qy * dz + qz * dy;
  C.E[2] = w * dy - dw * qy - qz * dx + qx * dz;
  C.E[3] = w * dz - dw * qz - qx * dy + qy * dx;
  const float rQ = rsqrt_sfu(dw * dw + dx * dx + dy * dy + dz * dz);
  C.s = copysignf(rQ, C.E[0]);  // sign fix folded into the normalisation
  C.qe[0] = C.s * C.E[0]; C.qe[1] = C.s * C.E[1]; C.qe[2] = C.s * C.E[2]; C.qe[3] = C.s * C.E[3];
  const float f0 = P.f0c * fh;
  float f1 = P.qa[0] * C.qe[1] - P.wa[0] * x[WX];
  float f2 = P.qa[1] * C.qe[2] - P.wa[1] * x[WX + 1];
  float f3 = P.qa[2] * C.qe[3] - P.wa[2] * x[WX + 2];
  if (PID) {
    // mix_i taumax_i (kI_i xi_i - kD_i omega'_i), added after the P term
    f1 = fmaf(-P.kdc[0], wdot[0], fmaf(P.kic[0], x[XI], f1));
    f2 = fmaf(-P.kdc[1], wdot[1], fmaf(P.kic[1], x[XI + 1], f2));
    f3 = fmaf(-P.kdc[2], wdot[2], fmaf(P.kic[2], x[XI + 2], f3));
#pragma unroll
    for (int i = 0; i < 3; ++i) e[i] = P.katt2[i] * C.qe[1 + i] - x[WX + i];
  }
  // G^-1: rotor i takes f0 + (+-f1) + (+-f2) + (+-f3); the last add saturates
  const float a = f0 + f1, d = f0 - f1, g3 = f3 - f2, h3 = f2 + f3;
  C.S[0] = a + g3;
  C.S[1] = d - h3;
  C.S[2] = d + h3;
  C.S[3] = a - g3;
  r[0] = sqrt_sfu(add_sat(a, g3));
  r[1] = sqrt_sfu(sub_sat(d, h3));
  r[2] = sqrt_sfu(add_sat(d, h3));
  r[3] = sqrt_sfu(sub_sat(a, g3));
}

__device__ __forceinline__ void controller(const DevGroup& P, const float* x, const float4 c, const Hd& hd,
                                           const float b[3], float r[4]) {
  Ctl C;
  controller_fwd(P, x, c, hd, b, C, r);
}

// ------------------------------------------------------------------ RK4 --
// One classical RK4 step with the rotor command held, from the first stage's
// rb_stage values at x (f1, dq1, dw1: omega' over the torque coefficients)
// and dOm = u - Omega.  The rotation and
// the rotor lag go through the four stages; the translation takes lin_coef's
// weights.  Each update is one product and one sum, written as the
// multiply-add it is.
__device__ __forceinline__ void rk4_from(const DevGroup& P, St& x, const float dOm[4], const StepH& H,
                                         const LinCoef& L, const float f1[3], const float dq1[4],
                                         const float dw1[3]) {
  float Om[4], q[4], w[3], aq[4], aw[3], f2[3], f3[3], f4[3], dq[4], dw[3], b[3];
#pragma unroll
  for (int i = 0; i < 4; ++i) { aq[i] = dq1[i]; q[i] = fmaf(H.h2q, dq1[i], x.a[QW + i]); }
#pragma unroll
  for (int i = 0; i < 3; ++i) { aw[i] = dw1[i]; w[i] = fmaf(L.t2[i], dw1[i], x.a[WX + i]); }
#pragma unroll
  for (int i = 0; i < 4; ++i) Om[i] = fmaf(L.c2, dOm[i], x.a[OM + i]);
  rb_stage(P, q, w, Om, f2, dq, dw, b);
#pragma unroll
  for (int i = 0; i < 4; ++i) { aq[i] = fmaf(2.f, dq[i], aq[i]); q[i] = fmaf(H.h2q, dq[i], x.a[QW + i]); }
#pragma unroll
  for (int i = 0; i < 3; ++i) { aw[i] = fmaf(2.f, dw[i], aw[i]); w[i] = fmaf(L.t2[i], dw[i], x.a[WX + i]); }
#pragma unroll
  for (int i = 0; i < 4; ++i) Om[i] = fmaf(L.c3, dOm[i], x.a[OM + i]);
  rb_stage(P, q, w, Om, f3, dq, dw, b);
#pragma unroll
  for (int i = 0; i < 4; ++i) { aq[i] = fmaf(2.f, dq[i], aq[i]); q[i] = fmaf(H.hq, dq[i], x.a[QW + i]); }
#pragma unroll
  for (int i = 0; i < 3; ++i) { aw[i] = fmaf(2.f, dw[i], aw[i]); w[i] = fmaf(L.t1[i], dw[i], x.a[WX + i]); }
#pragma unroll
  for (int i = 0; i < 4; ++i) Om[i] = fmaf(L.c4, dOm[i], x.a[OM + i]);
  rb_stage(P, q, w, Om, f4, dq, dw, b);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.a[QW + i] = fmaf(H.h6q, aq[i] + dq[i], x.a[QW + i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) x.a[WX + i] = fmaf(L.t6[i], aw[i] + dw[i], x.a[WX + i]);
#pragma unroll
  for (int i = 0; i < 4; ++i) x.a[OM + i] = fmaf(L.c5, dOm[i], x.a[OM + i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float v = x.a[VX + i];
    // gravity's share, a constant of the step, in the innermost term of z
    const float p3 = i == 2 ? fmaf(L.d3, f3[i], L.gd) : __fmul_rn(L.d3, f3[i]);
    const float v4 = i == 2 ? fmaf(L.b4, f4[i], L.gb) : __fmul_rn(L.b4, f4[i]);
    const float dp = fmaf(L.g, v, fmaf(L.d1, f1[i], fmaf(L.d2, f2[i], p3)));
    const float dv = fmaf(L.am1, v, fmaf(L.b1, f1[i], fmaf(L.b2, f2[i], fmaf(L.b3, f3[i], v4))));
    x.a[PX + i] = __fadd_rn(x.a[PX + i], dp);
    x.a[VX + i] = __fadd_rn(v, dv);
  }
}

template <int MODE>
__device__ __forceinline__ void step(const DevGroup& P, St& x, const float4 c, const Hd& hd, const StepH& H,
                                     const LinCoef& L) {
  // the first RK4 stage at x before the controller: the controller takes its
  // thrust axis, and the PID rate loop's derivative term its omega'
  float f[3], dq[4], dw[3], b[3], dOm[4];
  rb_stage(P, x.a + QW, x.a + WX, x.a + OM, f, dq, dw, b);
  if (MODE == 0) {
    dOm[0] = c.x - x.a[OM]; dOm[1] = c.y - x.a[OM + 1]; dOm[2] = c.z - x.a[OM + 2]; dOm[3] = c.w - x.a[OM + 3];
    rk4_from(P, x, dOm, H, L, f, dq, dw);
    return;
  }
  float r[4], e[3], wd[3];
  if (MODE == 2) {  // the derivative term takes omega' itself
    wd[0] = __fmul_rn(P.txc, dw[0]);
    wd[1] = __fmul_rn(P.tyc, dw[1]);
    wd[2] = __fmul_rn(P.tzc, dw[2]);
  }
  Ctl C;
  controller_fwd<MODE == 2>(P, x.a, c, hd, b, C, r, wd, e);
#pragma unroll
  for (int i = 0; i < 4; ++i) dOm[i] = fmaf(P.omax, r[i], -x.a[OM + i]);  // u = omega_max r
  rk4_from(P, x, dOm, H, L, f, dq, dw);
  if (MODE == 2) {
#pragma unroll
    for (int i = 0; i < 3; ++i) x.a[XI + i] = clampf(x.a[XI + i] + H.h * e[i], -P.xim[i], P.xim[i]);
  }
}

}  // namespace qs
