// Internal declarations shared by the host and device translation units of
// liblbm.so.  Not part of the public ABI (include/lbm.h is).
#pragma once

#include <cstddef>
#include <cstdint>

#include "../../include/lbm.h"

#ifdef __CUDACC__
#define LBM_HD __host__ __device__
#else
#define LBM_HD
#endif

namespace lbm {

constexpr int NPOP = 37;
constexpr int HALO = 3;
constexpr int NPAIR = 18;
constexpr int NSHELL = 8;   // |xi|^2 in {0,1,2,4,5,8,9,10}

// Representatives R_k of the (+R_k, -R_k) pairs, k = 0..17 (library order).
LBM_HD constexpr int rep_x(int k) {
  return k == 0 ? 1 : k == 1 ? 0 : k == 2 ? 1 : k == 3 ? -1 : k == 4 ? 2 : k == 5 ? 0 :
         k == 6 ? 2 : k == 7 ? 1 : k == 8 ? -1 : k == 9 ? -2 : k == 10 ? 2 : k == 11 ? -2 :
         k == 12 ? 3 : k == 13 ? 0 : k == 14 ? 3 : k == 15 ? 1 : k == 16 ? -1 : -3;
}
LBM_HD constexpr int rep_y(int k) {
  return k == 0 ? 0 : k == 1 ? 1 : k == 2 ? 1 : k == 3 ? 1 : k == 4 ? 0 : k == 5 ? 2 :
         k == 6 ? 1 : k == 7 ? 2 : k == 8 ? 2 : k == 9 ? 1 : k == 10 ? 2 : k == 11 ? 2 :
         k == 12 ? 0 : k == 13 ? 3 : k == 14 ? 1 : k == 15 ? 3 : k == 16 ? 3 : 1;
}
// Integer velocity xi_l of population l.
LBM_HD constexpr int vx(int l) { return l == 0 ? 0 : (l & 1) ? rep_x((l - 1) / 2) : -rep_x((l - 1) / 2); }
LBM_HD constexpr int vy(int l) { return l == 0 ? 0 : (l & 1) ? rep_y((l - 1) / 2) : -rep_y((l - 1) / 2); }
LBM_HD constexpr int sq(int l) { return vx(l) * vx(l) + vy(l) * vy(l); }
// Shell index 0..7 of |xi|^2 = 0,1,2,4,5,8,9,10.
LBM_HD constexpr int shell_index(int s) {
  return s == 0 ? 0 : s == 1 ? 1 : s == 2 ? 2 : s == 4 ? 3 : s == 5 ? 4 : s == 8 ? 5 : s == 9 ? 6 : 7;
}
LBM_HD constexpr int shell_sq(int j) {
  return j == 0 ? 0 : j == 1 ? 1 : j == 2 ? 2 : j == 3 ? 4 : j == 4 ? 5 : j == 5 ? 8 : j == 6 ? 9 : 10;
}
LBM_HD constexpr int pair_shell(int k) { return shell_index(rep_x(k) * rep_x(k) + rep_y(k) * rep_y(k)); }

// Host-derived float64 constants of the D2Q37 quadrature.
struct Quadrature {
  double r;            // c_l = r xi_l
  double y;            // 1 / r^2
  double w_shell[NSHELL];
  double c2_shell[NSHELL];  // r^2 |xi|^2, rounded from a double-double value
  double w[NPOP];
  double w_shell_lo[NSHELL];  // low parts of the double-double weights
  double y_lo;
};

// Solve the isotropy conditions in double-double arithmetic (quadrature.cpp).
// Returns 0 on success, else writes a message into err.
int solve_quadrature(Quadrature* out, char* err, size_t errlen);
// Wall ratios q_l = phi_l / sum over the wall's 26 unknown slots of phi, with
// phi_l = f^eq_l(1, 0, T_wall); wall = 0 bottom, 1 top.  Zero for l that is
// not an unknown of that wall.
void wall_ratios(const Quadrature& q, double t_wall, int wall, double out[NPOP]);
// Inverse Gram blocks of the weighted velocity monomials for the regularised
// collide (quadrature.cpp).  Returns 0 on success.
int regularization_gram_inverse(const Quadrature& q, double out[63]);

// Per-launch constants of a lattice, passed by value (kernel parameter space).
struct LatticeArgs {
  int lx, ly;
  long long plane;       // (ly + 6) * lx elements per population plane
  int periodic_y;
  double omega;          // 1 / tau
  double omc;            // 1 - omega
  double r;              // c_l = r xi_l
  double r2;             // r^2
  double inv_r2;         // 1 / r^2
  double tau_g_xi;       // tau g / r: the gravity shift of u in xi units
  double tshift;         // tau (1 - tau) g^2 / D - 1: theta = T + tshift
  double tau;
  double g;              // gravity magnitude (along -y)
  double rho0;           // FP32 shift density
  double w_shell[NSHELL];
  double c2_shell[NSHELL];
  // per-shell multiples for the float64 collide: c2 / 2, c2 / 4, c2^2 / 8, w / 6
  double c2h_shell[NSHELL];
  double c2q_shell[NSHELL];
  double c4e_shell[NSHELL];
  double w6_shell[NSHELL];
  double q_bot[NPOP];
  double q_top[NPOP];
  float w_rho0_f[NPOP];  // w_l rho0 as float (FP32 decode of bc inputs)
  double w_rho0[NPOP];   // w_l rho0
  // float32 / double-float copies for the FP32-store collide
  float w_shell_f[NSHELL];
  float c2_shell_f[NSHELL];
  float omega_f, omc_f;
  float df_rho0[2];       // rho0
  float df_e0[2];         // D rho0 / r^2: sum_l w_l |xi_l|^2 rho0
  float df_r2[2];         // r^2
  float df_half_r2[2];    // r^2 / 2
  float df_inv_r2[2];     // 1 / r^2
  float df_tshift[2];     // tau (1 - tau) g^2 / D - 1
  float df_taug_r[2];     // tau g / r
  float df_g_r[2];        // g / r
  float df_omega[2];      // omega
  float df_omc[2];        // 1 - omega
  float df_w_shell[NSHELL][2];
  int regularized;        // LBM_FLAG_REGULARIZED
  double ginv[63];        // (1 - omega) x inverse Gram blocks EE(36) OE(9) EO(9) OO(9)
  float df_c2_shell[NSHELL][2];
  unsigned int* status;  // device status word
  // Site-relative offsets for states of fewer than 2^31 elements
  // (idx32 != 0), in bytes of the lattice's storage type: the pull source of
  // population l of an interior column lies pull_off[l] bytes from the site's
  // element in plane 0, its destination plane_off[l] bytes from it.  Whole
  // 64-bit byte offsets let every access add a kernel parameter to one
  // per-thread pointer, with no per-access widening or scaling.
  int idx32;
  int tma_loads;              // LBM_FLAG_TMA_LOADS
  long long pull_off[NPOP];   // (l plane - xi_ly lx - xi_lx) * element size
  long long plane_off[NPOP];  // l plane * element size
  // Arithmetic of the LBM_FP32_SHIFTED collide: FP32_ARITH_SPLIT (default),
  // FP32_ARITH_F64_TERMS (LBM_FLAG_FP32_F64_TERMS) or FP32_ARITH_F64_COLLIDE
  // (LBM_FLAG_FP32_F64_COLLIDE).
  int fp32_arith;
  double ow_shell[NSHELL];    // omega w_j
  // Exact sums of the shift constants w_rho0[l] (rho) and |xi_l|^2 w_rho0[l]
  // (Exi) as 96-bit two's-complement fixed point on the 2^-82 grid (words
  // w0, w1, w2); the momentum sums of the shift vanish exactly (+- pairs).
  unsigned fix_shift_rho[3];
  unsigned fix_shift_exi[3];
  // multiples of r^2 and r^4 in the monomial coefficients of the equilibrium
  double r2_2, r2_4, r4_4, r4_8;  // r^2 / 2, r^2 / 4, r^4 / 4, r^4 / 8
  double r2_tau_g_xi;  // r^2 tau_g_xi
  double tshift_v;     // tshift - (r^2 / 2) tau_g_xi^2
  double half_inv_r2;  // 1 / (2 r^2)
  double quarter_inv_r2;  // 1 / (4 r^2)
  double inv_r;         // 1 / r
  double uy_obs_shift;  // tau g - g / 2
};

enum { FP32_ARITH_SPLIT = 0, FP32_ARITH_F64_TERMS = 1, FP32_ARITH_F64_COLLIDE = 2 };

}  // namespace lbm
