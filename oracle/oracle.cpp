// TEST INFRASTRUCTURE ONLY: C entry points of the FP64 checker (built into
// oracle/liboracle.so).  Used by tests, the smoke check and the bench's CPU
// baseline; never by the CUDA library.
//
// Layouts: states are agent-major (n x 17 doubles: p v q omega Omega; n x 20
// in the PID mode, with the rate-error integral xi last), commands n x 4,
// parameter groups n_groups x 43 doubles in the packed order of
// unpack_group(), group ids int32.  Groups of car or fixed-wing type
// (vehicles.hpp) run their own model in the closed-loop mode.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#include "quad_model.hpp"
#include "vehicles.hpp"

namespace orc {
thread_local Tape* g_tape = nullptr;
thread_local OpCount g_count;
}  // namespace orc

using namespace orc;

namespace {

template <class F>
void parallel_for(int64_t n, int nthreads, F&& body) {
  if (nthreads <= 1 || n < 2) {
    body(0, n);
    return;
  }
  nthreads = (int)std::min<int64_t>(nthreads, n);
  std::vector<std::thread> pool;
  const int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    const int64_t lo = t * chunk, hi = std::min<int64_t>(n, lo + chunk);
    if (lo >= hi) break;
    pool.emplace_back([&body, lo, hi] { body(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

struct GroupSet {
  std::vector<Group<double>> P;
  std::vector<Fixed> F;
  GroupSet(const double* packed, int n_groups) {
    for (int g = 0; g < n_groups; ++g) {
      P.push_back(unpack_group(packed + (int64_t)g * NPARAM));
      F.push_back(make_fixed(P.back()));
    }
  }
};

// Running cost term of one step end: sum_i Omega_i^2.
inline double omega_sq(const double* x) {
  return x[13] * x[13] + x[14] * x[14] + x[15] * x[15] + x[16] * x[16];
}

}  // namespace

extern "C" {

int oracle_nparam() { return NPARAM; }

// Allocation matrix of Eq. 3 (row-major 4x4), its inverse and the per-axis
// torque limits for one packed parameter group.
int oracle_allocation(const double* group, double* G, double* Ginv, double* taumax) {
  const Fixed F = make_fixed(unpack_group(group));
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      G[i * 4 + j] = F.G[i][j];
      Ginv[i * 4 + j] = F.Ginv[i][j];
    }
  for (int i = 0; i < 3; ++i) taumax[i] = F.taumax[i];
  return 0;
}

// dx = f(x, w) for one agent.
int oracle_derivative(const double* group, const double* x, const double* w, double* dx) {
  const Group<double> P = unpack_group(group);
  const Fixed F = make_fixed(P);
  derivative(P, F, x, w, dx);
  return 0;
}

// Rotor-speed commands of the cascaded controller for one agent.
int oracle_controller(const double* group, const double* x, const double* cmd, double* w) {
  const Group<double> P = unpack_group(group);
  const Fixed F = make_fixed(P);
  controller(P, F, x, cmd, w);
  return 0;
}

// Distance of each car or fixed-wing agent's trajectory from its controller's
// one discontinuity, minimised over the nsteps step starts: for a fixed-wing
// drone pi - |course error| (atan2 jumps from +pi to -pi when the waypoint
// passes straight behind); for a car and a quadrotor +inf (pure pursuit is
// continuous in the state).  Trajectories that pass within rounding of the
// jump may take the other branch in another precision.
int oracle_vehicle_margins(const double* groups, int n_groups, const int32_t* gid, int64_t n, const double* x0,
                           const double* cmd, double h, int64_t nsteps, int nthreads, double* out) {
  if (n < 0 || nsteps < 0 || n_groups < 1) return -1;
  const GroupSet S(groups, n_groups);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t a = lo; a < hi; ++a) {
      const int g = gid ? gid[a] : 0;
      const Group<double>& P = S.P[g];
      double m = 1e300;
      if (P.type == TYPE_FIXED_WING) {
        double cur[NX], nxt[NX];
        std::memcpy(cur, x0 + a * NX, sizeof(cur));
        const double* c = cmd + a * 4;
        for (int64_t s = 0; s < nsteps; ++s) {
          const double dx = c[0] - cur[0], dy = c[1] - cur[1];
          const double cross = cur[6] * dy - cur[7] * dx, dot = cur[6] * dx + cur[7] * dy;
          m = std::min(m, M_PI - std::fabs(std::atan2(cross, dot)));
          vehicle_step(P, cur, c, h, nxt);
          std::memcpy(cur, nxt, sizeof(cur));
        }
      }
      out[a] = m;
    }
  });
  return 0;
}

// Car or fixed-wing agent: inputs u (3) of its controller at state x (17).
int oracle_vehicle_controller(const double* group, const double* x, const double* cmd, double* u) {
  const Group<double> P = unpack_group(group);
  if (P.type != TYPE_CAR && P.type != TYPE_FIXED_WING) return -1;
  vehicle_controller(P, x, cmd, u);
  return 0;
}

// Car or fixed-wing agent: time derivative (17) at state x for inputs u.
int oracle_vehicle_derivative(const double* group, const double* x, const double* u, double* dx) {
  const Group<double> P = unpack_group(group);
  if (P.type != TYPE_CAR && P.type != TYPE_FIXED_WING) return -1;
  vehicle_derivative(P, x, u, dx);
  return 0;
}

// PID mode, one agent with its 20-state x: rotor-speed commands w (4), the
// rate error e (3) and omega' at x (3), as the step uses them.
int oracle_controller_pid(const double* group, const double* x, const double* cmd, double* w, double* e,
                          double* wdot) {
  const Group<double> P = unpack_group(group);
  const Fixed F = make_fixed(P);
  double d0[NX];
  derivative(P, F, x, x + 13, d0);
  for (int i = 0; i < 3; ++i) wdot[i] = d0[10 + i];
  controller(P, F, x, cmd, w, nullptr, nullptr, x + NX, d0 + 10, e);
  return 0;
}

// Unit quaternion of a row-major 3x3 rotation matrix (Shepperd).
int oracle_shepperd(const double* R9, double* q) {
  double R[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R[i][j] = R9[i * 3 + j];
  shepperd(R, q);
  return 0;
}

// Advance n agents by nsteps RK4 steps of length h in place.  run_cost (may
// be NULL) receives, per agent, sum over step ends n = 1..nsteps of
// sum_i Omega_i^2.
int oracle_rollout(const double* groups, int n_groups, const int32_t* gid, int64_t n, double* x,
                   const double* cmd, double h, int64_t nsteps, int mode, int nthreads, double* run_cost) {
  if (n < 0 || nsteps < 0 || n_groups < 1 || mode < OPEN_LOOP || mode > CLOSED_LOOP_PID) return -1;
  const GroupSet S(groups, n_groups);
  for (int g = 0; g < n_groups; ++g)
    if (S.P[g].type != TYPE_QUAD && (S.P[g].type > TYPE_FIXED_WING || mode != CLOSED_LOOP)) return -1;
  const int nx = state_dim(mode);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t a = lo; a < hi; ++a) {
      const int g = gid ? gid[a] : 0;
      double cur[NXP], nxt[NXP];
      std::memcpy(cur, x + a * nx, nx * sizeof(double));
      double rc = 0.0;
      for (int64_t s = 0; s < nsteps; ++s) {
        agent_step(S.P[g], S.F[g], mode, cur, cmd + a * 4, h, nxt);
        std::memcpy(cur, nxt, nx * sizeof(double));
        rc += omega_sq(cur);
      }
      std::memcpy(x + a * nx, cur, nx * sizeof(double));
      if (run_cost) run_cost[a] = rc;
    }
  });
  return 0;
}

// The same rollout of quadrotor groups evaluated in FP32: the model above
// instantiated on float, every operation rounded to single precision (the
// library is compiled without contraction), the state stored as float between
// steps.  Its distance from the FP64 rollout is what FP32 rounding alone does
// to these equations over nsteps steps; tests use it to size the bar of the
// FP32 CUDA path beyond the stated 1000-step one.  x is n x state_dim floats.
int oracle_rollout_f32(const double* groups, int n_groups, const int32_t* gid, int64_t n, float* x,
                       const double* cmd, double h, int64_t nsteps, int mode, int nthreads) {
  if (n < 0 || nsteps < 0 || n_groups < 1 || mode < OPEN_LOOP || mode > CLOSED_LOOP_PID) return -1;
  const GroupSet S(groups, n_groups);
  std::vector<Group<float>> P32;
  for (int g = 0; g < n_groups; ++g) {
    if (S.P[g].type != TYPE_QUAD) return -1;
    P32.push_back(cast_group<float>(S.P[g]));
  }
  const int nx = state_dim(mode);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t a = lo; a < hi; ++a) {
      const int g = gid ? gid[a] : 0;
      float cur[NXP], nxt[NXP];
      std::memcpy(cur, x + a * nx, nx * sizeof(float));
      for (int64_t s = 0; s < nsteps; ++s) {
        step_any(P32[g], S.F[g], mode, cur, cmd + a * 4, h, nxt);
        std::memcpy(cur, nxt, nx * sizeof(float));
      }
      std::memcpy(x + a * nx, cur, nx * sizeof(float));
    }
  });
  return 0;
}

// Per-agent loss L_a = |p_T - goal_a|^2 + w_omega * sum_{n=1..T} sum_i Omega_{n,i}^2
// and its exact discrete gradient by reverse mode: dL/dx0 (n x 17; n x 20 in
// the PID mode) and
// dL/dtheta (n x 16, order kp kd katt krate m Jxx Jyy Jzz) of the agent's
// own group parameters.  The forward states are stored; each step is then
// re-taped on its own and swept backwards with the incoming adjoint.
int oracle_grad(const double* groups, int n_groups, const int32_t* gid, int64_t n, const double* x0,
                const double* cmd, double h, int64_t nsteps, int mode, const double* goal, double w_omega,
                int nthreads, double* loss, double* dx0, double* dtheta) {
  if (n < 0 || nsteps < 0 || n_groups < 1 || mode < OPEN_LOOP || mode > CLOSED_LOOP_PID) return -1;
  const GroupSet S(groups, n_groups);
  for (int g = 0; g < n_groups; ++g)
    if (S.P[g].type != TYPE_QUAD) return -1;  // quadrotor gradients only
  const int NS = state_dim(mode);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    Tape tape;
    g_tape = &tape;
    std::vector<double> xs((nsteps + 1) * NS);
    std::vector<double> adj;
    for (int64_t a = lo; a < hi; ++a) {
      const int g = gid ? gid[a] : 0;
      const Group<double>& Pd = S.P[g];
      const Fixed& F = S.F[g];
      const double* c = cmd + a * 4;
      std::memcpy(xs.data(), x0 + a * NS, NS * sizeof(double));
      double rc = 0.0;
      for (int64_t s = 0; s < nsteps; ++s) {
        step_any(Pd, F, mode, xs.data() + s * NS, c, h, xs.data() + (s + 1) * NS);
        rc += omega_sq(xs.data() + (s + 1) * NS);
      }
      const double* xT = xs.data() + nsteps * NS;
      double L = w_omega * rc;
      double lam[NXP] = {0};
      for (int i = 0; i < 3; ++i) {
        const double d = xT[i] - goal[a * 3 + i];
        L += d * d;
        lam[i] = 2.0 * d;
      }
      if (nsteps > 0)
        for (int i = 0; i < 4; ++i) lam[13 + i] = 2.0 * w_omega * xT[13 + i];
      double th[NTHETA] = {0};
      for (int64_t s = nsteps - 1; s >= 0; --s) {
        tape.clear();
        Group<Var> Pv = cast_group<Var>(Pd);
        for (int i = 0; i < 3; ++i) Pv.kp[i] = Var::leaf(Pd.kp[i]);
        for (int i = 0; i < 3; ++i) Pv.kd[i] = Var::leaf(Pd.kd[i]);
        for (int i = 0; i < 3; ++i) Pv.katt[i] = Var::leaf(Pd.katt[i]);
        for (int i = 0; i < 3; ++i) Pv.krate[i] = Var::leaf(Pd.krate[i]);
        Pv.m = Var::leaf(Pd.m);
        for (int i = 0; i < 3; ++i) Pv.J[i] = Var::leaf(Pd.J[i]);
        Var xv[NXP], xn[NXP];
        for (int i = 0; i < NS; ++i) xv[i] = Var::leaf(xs[s * NS + i]);
        step_any(Pv, F, mode, xv, c, h, xn);
        adj.assign(tape.nodes.size(), 0.0);
        for (int i = 0; i < NS; ++i)
          if (xn[i].idx >= 0) adj[xn[i].idx] += lam[i];
        tape.backprop(adj);
        // theta leaves were created first, in theta order (indices 0..15)
        for (int k = 0; k < NTHETA; ++k) th[k] += adj[k];
        for (int i = 0; i < NS; ++i) lam[i] = adj[xv[i].idx];
        if (s >= 1)
          for (int i = 0; i < 4; ++i) lam[13 + i] += 2.0 * w_omega * xs[s * NS + 13 + i];
      }
      loss[a] = L;
      if (dx0) std::memcpy(dx0 + a * NS, lam, NS * sizeof(double));
      if (dtheta) std::memcpy(dtheta + a * NTHETA, th, sizeof(th));
    }
    g_tape = nullptr;
  });
  return 0;
}

// Distance of each agent's closed-loop trajectory from the kinks of the
// controller, minimised over the nsteps step starts: out[a*3 + 0] = min over
// rotors of |S_i| / omega_max^2 (S = unclamped Omega_cmd^2; sqrt has an
// unbounded derivative at 0), out[a*3 + 1] = min |S_i - omega_max^2| /
// omega_max^2 (rotor ceiling), out[a*3 + 2] = min ||ar_i| - a_max| / a_max
// (acceleration clamp; in the PID mode also the integrator clamp,
// min ||xi_i + h e_i| - xi_max| / xi_max).  Gradients of agents with a small margin are
// ill-conditioned: a perturbation at rounding level moves them by a finite
// amount.
int oracle_clamp_margins(const double* groups, int n_groups, const int32_t* gid, int64_t n, const double* x0,
                         const double* cmd, double h, int64_t nsteps, int mode, int nthreads, double* out) {
  if (n < 0 || nsteps < 0 || n_groups < 1 || (mode != CLOSED_LOOP && mode != CLOSED_LOOP_PID)) return -1;
  const GroupSet S(groups, n_groups);
  for (int g = 0; g < n_groups; ++g)
    if (S.P[g].type != TYPE_QUAD) return -1;
  const int nx = state_dim(mode);
  parallel_for(n, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t a = lo; a < hi; ++a) {
      const int g = gid ? gid[a] : 0;
      const Group<double>& P = S.P[g];
      double cur[NXP], nxt[NXP];
      std::memcpy(cur, x0 + a * nx, nx * sizeof(double));
      const double om2 = P.omega_max * P.omega_max;
      double m0 = 1e300, m1 = 1e300, m2 = 1e300;
      for (int64_t s = 0; s < nsteps; ++s) {
        double ar[3], Sd[4], w[4];
        if (mode == CLOSED_LOOP_PID) {
          double d0[NX], e[3];
          derivative(P, S.F[g], cur, cur + 13, d0);
          controller(P, S.F[g], cur, cmd + a * 4, w, ar, Sd, cur + NX, d0 + 10, e);
          // the integrator clamp is a kink of the same kind as the acceleration clamp
          for (int i = 0; i < 3; ++i)
            if (P.xi_max[i] > 0.0)
              m2 = std::min(m2, std::fabs(std::fabs(cur[NX + i] + h * e[i]) - P.xi_max[i]) / P.xi_max[i]);
        } else {
          controller(P, S.F[g], cur, cmd + a * 4, w, ar, Sd);
        }
        for (int i = 0; i < 4; ++i) {
          m0 = std::min(m0, std::fabs(Sd[i]) / om2);
          m1 = std::min(m1, std::fabs(Sd[i] - om2) / om2);
        }
        for (int i = 0; i < 3; ++i) m2 = std::min(m2, std::fabs(std::fabs(ar[i]) - P.a_max) / P.a_max);
        step_any(P, S.F[g], mode, cur, cmd + a * 4, h, nxt);
        std::memcpy(cur, nxt, nx * sizeof(double));
      }
      out[a * 3 + 0] = m0;
      out[a * 3 + 1] = m1;
      out[a * 3 + 2] = m2;
    }
  });
  return 0;
}

// Collision test of one ordered pair, as a plain definition: live agents i
// and j (i != j) collide when their centres are closer than the sum of their
// bounding radii.  The decision is taken in FP32 with every operation rounded
// on its own (the checker is built without floating contraction): dx = p_j - p_i per axis,
// d2 = (dx*dx + dy*dy) + dz*dz, thr = (r_i + r_j)^2, collide if d2 < thr.
static inline bool pair_collides(const float* pi, float ri, const float* pj, float rj) {
  const float dx = pj[0] - pi[0], dy = pj[1] - pi[1], dz = pj[2] - pi[2];
  const float xx = dx * dx, yy = dy * dy, zz = dz * dz;
  const float s = xx + yy;
  const float d2 = s + zz;
  const float rs = ri + rj;
  const float thr = rs * rs;
  return d2 < thr;
}

// Marks hit[a] = 1 for every live agent a (alive[a] != 0) that collides with
// another live agent, by brute force over all pairs (Sec. III-A: colliding
// agents are marked dead and excluded).  p: n x 3 float positions; radius:
// n floats.  With m >= 0 and idx given, only agents idx[0..m) are decided
// (each against all n), and hit is indexed like idx.
int oracle_collisions(const float* p, const float* radius, const uint8_t* alive, int64_t n, const int64_t* idx,
                      int64_t m, int nthreads, uint8_t* hit) {
  if (n < 0) return -1;
  const int64_t count = idx ? m : n;
  parallel_for(count, nthreads, [&](int64_t lo, int64_t hi) {
    for (int64_t k = lo; k < hi; ++k) {
      const int64_t a = idx ? idx[k] : k;
      uint8_t h = 0;
      if (alive[a]) {
        for (int64_t b = 0; b < n && !h; ++b) {
          if (b == a || !alive[b]) continue;
          if (pair_collides(p + 3 * a, radius[a], p + 3 * b, radius[b])) h = 1;
        }
      }
      hit[k] = h;
    }
  });
  return 0;
}

// Reverse-sweep work of one step in the checker's reverse mode: the number of
// tape edges of a step (any mode) taped with respect to its states and the 16
// differentiated parameters.  Sweeping backwards costs one
// multiply and one add per edge.
int oracle_count_adjoint_edges(const double* group, const double* x, const double* cmd, double h, int mode,
                               int64_t* edges) {
  const Group<double> Pd = unpack_group(group);
  const Fixed F = make_fixed(Pd);
  Tape tape;
  g_tape = &tape;
  Group<Var> Pv = cast_group<Var>(Pd);
  for (int i = 0; i < 3; ++i) {
    Pv.kp[i] = Var::leaf(Pd.kp[i]);
    Pv.kd[i] = Var::leaf(Pd.kd[i]);
    Pv.katt[i] = Var::leaf(Pd.katt[i]);
    Pv.krate[i] = Var::leaf(Pd.krate[i]);
    Pv.J[i] = Var::leaf(Pd.J[i]);
  }
  Pv.m = Var::leaf(Pd.m);
  Var xv[NXP], xn[NXP];
  for (int i = 0; i < state_dim(mode); ++i) xv[i] = Var::leaf(x[i]);
  step_any(Pv, F, mode, xv, cmd, h, xn);
  int64_t e = 0;
  for (const Node& n : tape.nodes) e += (n.a >= 0) + (n.b >= 0);
  *edges = e;
  g_tape = nullptr;
  return 0;
}

// Non-trivial FP64 operations of one evaluation of the time derivative (the
// 17 states, rotor commands w): the PID step evaluates it once more for
// omega', which a step implementation may take from its first RK4 stage.
int oracle_count_derivative_ops(const double* group, const double* x, const double* w, int64_t* counts) {
  const Group<double> Pd = unpack_group(group);
  const Fixed F = make_fixed(Pd);
  const Group<Cnt> P = cast_group<Cnt>(Pd);
  Cnt xc[NX], wc[4], dx[NX];
  for (int i = 0; i < NX; ++i) xc[i] = Cnt(x[i]);
  for (int i = 0; i < 4; ++i) wc[i] = Cnt(w[i]);
  g_count = OpCount();
  derivative(P, F, xc, wc, dx);
  counts[0] = g_count.add;
  counts[1] = g_count.mul;
  counts[2] = g_count.div;
  counts[3] = g_count.sqrt;
  counts[4] = g_count.trig;
  counts[5] = g_count.cmp;
  return 0;
}

// Non-trivial FP64 operations of one step for one agent:
// counts = {add/sub, mul, div, sqrt, sin/cos, comparisons}.
int oracle_count_ops(const double* group, const double* x, const double* cmd, double h, int mode,
                     int64_t* counts) {
  const Group<double> Pd = unpack_group(group);
  const Fixed F = make_fixed(Pd);
  const Group<Cnt> P = cast_group<Cnt>(Pd);
  Cnt xc[NXP], xn[NXP];
  for (int i = 0; i < state_dim(mode); ++i) xc[i] = Cnt(x[i]);
  g_count = OpCount();
  agent_step(P, F, mode, xc, cmd, h, xn);
  counts[0] = g_count.add;
  counts[1] = g_count.mul;
  counts[2] = g_count.div;
  counts[3] = g_count.sqrt;
  counts[4] = g_count.trig;
  counts[5] = g_count.cmp;
  return 0;
}

}  // extern "C"
