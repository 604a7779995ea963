// Grad-13 wall flux of the synthetic solve (Section 3.3, Eqs. G13_VDF and GSIS-DVM-flux).
//
// Units as everywhere in the library: velocity in sqrt(2 R T0), p = rho T / 2, the stress
// sigma = int c c f - p I, the translational heat flux q_t = int c^2 c f / 2 and the rotational
// one q_r = int c f1.  The 13-moment VDF with these moments is
//   f0 = M [1 + A:cc + (B.c)(c^2/T - 5/2)],  A = 2 sigma / (rho T^2),  B = 8 q_t / (5 rho T^2),
//   f1 = (d_r T_r / 4) f0 + 2 M (q_r.c) / (rho T),
// M the Maxwellian of (rho, u, T_t).  The gas moving into the wall (xi.n > 0, n the outward unit
// normal) carries it; the wall re-emits rho_w M(u_w, T_w) with zero net mass flux.
//
// Integrating over the face's tangential plane in closed form leaves one-dimensional integrals
// of polynomials in x = c.n against the half-range moments
//   H_k = int_{x > -u_n} x^k g(x) dx,  g the Maxwellian of variance T/2,
//   H_0 = erfc(-u_n / sqrt T) / 2,  H_k = (k-1) (T/2) H_{k-2} + (T/2) (-u_n)^(k-1) g(-u_n),
// and the tangential averages of f0 / M are
//   <Q>         = 1 - A_nn T/2 - (3/2) B_n x + A_nn x^2 + (B_n / T) x^3,
//   <c_t Q>     = -(T/4) B_t + T A_nt x + (1/2) B_t x^2,
//   <|c_t|^2 Q> = T - A_nn T^2 - (T/2) B_n x + A_nn T x^2 + B_n x^3,
// with A_nn = n.A.n and A_nt, B_t the tangential parts of A n and B.  Every flux is then a sum
// of LH_k = int (u_n + x) x^k g = u_n H_k + H_{k+1}.
#pragma once

namespace gsis {

// F: outward flux per unit area of mass, momentum (3), total energy and (Rykov, nW = 6)
// rotational energy; sig6 = (xx yy zz xy xz yz); uw, Tw: the wall (uw tangential to it).
__device__ __forceinline__ void grad13_wall_flux(int nW, double d_r, double rho, const double *u, double T,
                                                 double Tr, const double *n, const double *sig6, const double *qt,
                                                 const double *qr, const double *uw, double Tw, double *F) {
  const double kPi_ = 3.14159265358979323846;
  const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
  // sigma n, its normal and tangential parts; the heat flux likewise
  const double sn0 = sig6[0] * n[0] + sig6[3] * n[1] + sig6[4] * n[2];
  const double sn1 = sig6[3] * n[0] + sig6[1] * n[1] + sig6[5] * n[2];
  const double sn2 = sig6[4] * n[0] + sig6[5] * n[1] + sig6[2] * n[2];
  const double snn = sn0 * n[0] + sn1 * n[1] + sn2 * n[2];
  const double qn = qt[0] * n[0] + qt[1] * n[1] + qt[2] * n[2];
  const double iA = 2.0 / (rho * T * T), iB = 1.6 / (rho * T * T);
  const double Ann = iA * snn, Bn = iB * qn;
  const double sn[3] = {sn0, sn1, sn2};
  double Ant[3], Bt[3], ut[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Ant[a] = iA * (sn[a] - snn * n[a]);
    Bt[a] = iB * (qt[a] - qn * n[a]);
    ut[a] = u[a] - un * n[a];
  }
  // half-range moments H_0 .. H_6 and LH_0 .. LH_5
  const double sr = un / sqrt(T), g0 = exp(-sr * sr) / sqrt(kPi_ * T), hT = 0.5 * T;
  double H[7];
  H[0] = 0.5 * erfc(-sr);
  H[1] = hT * g0;
  double pw = -un;  // (-u_n)^(k-1), from k = 2
#pragma unroll
  for (int k = 2; k < 7; ++k) {
    H[k] = (k - 1) * hT * H[k - 2] + hT * pw * g0;
    pw *= -un;
  }
  double LH[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) LH[k] = un * H[k] + H[k + 1];
  const double q[4] = {1.0 - 0.5 * Ann * T, -1.5 * Bn, Ann, Bn / T};
  const double r[4] = {T - Ann * T * T, -0.5 * Bn * T, Ann * T, Bn};
  const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  double mass = 0.0, normal = 0.0, energy = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    mass += q[k] * LH[k];
    normal += q[k] * (un * LH[k] + LH[k + 1]);
    energy += q[k] * (0.5 * u2 * LH[k] + un * LH[k + 1] + 0.5 * LH[k + 2]) + 0.5 * r[k] * LH[k];
  }
  // <c_t Q> = t0 + t1 x + t2 x^2 (vectors)
  double tang[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double t0 = -0.25 * T * Bt[a], t1 = T * Ant[a], t2 = 0.5 * Bt[a];
    const double lt = t0 * LH[0] + t1 * LH[1] + t2 * LH[2];
    tang[a] = ut[a] * mass + lt;
    energy += ut[a] * lt;
  }
  double rot = 0.0;
  if (nW == 6) {
    const double qrn = qr[0] * n[0] + qr[1] * n[1] + qr[2] * n[2];
    rot = d_r * Tr / 4.0 * mass + 2.0 * qrn / (rho * T) * LH[1];
  }
  // the wall's half
  const double K1 = -sqrt(Tw) / (2.0 * sqrt(kPi_)), K2 = Tw / 4.0, K3 = Tw * K1;
  const double rw = -rho * mass / K1;
  const double uwn = uw[0] * n[0] + uw[1] * n[1] + uw[2] * n[2];
  double uwt[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) uwt[a] = uw[a] - uwn * n[a];
  const double uw2 = uwt[0] * uwt[0] + uwt[1] * uwt[1] + uwt[2] * uwt[2];
  F[0] = rho * mass + rw * K1;
#pragma unroll
  for (int a = 0; a < 3; ++a) F[1 + a] = rho * (n[a] * normal + tang[a]) + n[a] * rw * K2 + rw * K1 * uwt[a];
  const double rin = rho * rot, rout = nW == 6 ? d_r * Tw / 4.0 * rw * K1 : 0.0;
  F[4] = rho * energy + rin + 0.5 * rw * (K3 + K1 * (uw2 + Tw)) + rout;
  F[5] = rin + rout;
}

}  // namespace gsis
