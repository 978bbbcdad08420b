// Device geometry of the coarse and fine MFS discretizations (FP64).
// Global frame, counterclockwise, angle 0 along +x.
#pragma once
#include <cmath>

#include "lmfs_internal.h"

namespace lmfs {

struct PairFrame {
  double c1x, c1y, c2x, c2y, r1, r2;
  double d, cphi, sphi;   // centre distance and direction c1 -> c2
  double p1, p2;          // limiting-point distances from c1 and c2
};

// Limiting points of two circles: where successive image reflections
// accumulate (Sec. 5: R_acc(delta) = 1 + delta/2 - sqrt(delta + delta^2/4) for
// unit disks).  Unequal radii: smaller root of d p^2 - (d^2 + r1^2 - r2^2) p +
// d r1^2 = 0.
__host__ __device__ inline PairFrame make_frame(double c1x, double c1y, double r1, double c2x,
                                                double c2y, double r2) {
  PairFrame f;
  f.c1x = c1x; f.c1y = c1y; f.c2x = c2x; f.c2y = c2y; f.r1 = r1; f.r2 = r2;
  const double dx = c2x - c1x, dy = c2y - c1y;
  f.d = sqrt(dx * dx + dy * dy);
  f.cphi = dx / f.d;
  f.sphi = dy / f.d;
  const double a = f.d * f.d + r1 * r1 - r2 * r2;
  f.p1 = (a - sqrt(fmax(a * a - 4.0 * f.d * f.d * r1 * r1, 0.0))) / (2.0 * f.d);
  const double b = f.d * f.d + r2 * r2 - r1 * r1;
  f.p2 = (b - sqrt(fmax(b * b - 4.0 * f.d * f.d * r2 * r2, 0.0))) / (2.0 * f.d);
  return f;
}

// Shielding ellipse node j (0 <= j < 2 N_ell) in body-local complex
// coordinates (Sec. 5): z = a/2 [1 + cos(theta + i alpha)],
// alpha = arccosh(1 + 2 gamma (rad - a)/a), theta_j = (j + 1/2) pi / N_ell.
// Returns false if |z| <= rad * Rf (node dropped).
__host__ __device__ inline bool ellipse_node(double a, double rad, double Rf, int Nell, double gamma,
                                             int j, double* zr, double* zi) {
  const double alpha = acosh(1.0 + 2.0 * gamma * (rad - a) / a);
  const double th = (j + 0.5) * LMFS_PI / Nell;
  // cos(th + i alpha) = cos th cosh alpha - i sin th sinh alpha
  *zr = 0.5 * a * (1.0 + cos(th) * cosh(alpha));
  *zi = -0.5 * a * sin(th) * sinh(alpha);
  return sqrt((*zr) * (*zr) + (*zi) * (*zi)) > rad * Rf;
}

// Pair-adapted node angle (Sec. 5): theta = 2 pi j / M,
// theta~ = pi + arg((e^{i theta} + r)/(1 + r e^{i theta})).
__host__ __device__ inline double mobius_angle(int j, int M, double r) {
  const double th = 2.0 * LMFS_PI * j / M;
  const double c = cos(th), s = sin(th);
  // (c + r + i s) / (1 + r c + i r s)
  const double nr = c + r, ni = s, dr = 1.0 + r * c, di = r * s;
  const double qr = nr * dr + ni * di, qi = ni * dr - nr * di;
  return LMFS_PI + atan2(qi, qr);
}

// Peanut node p of M_p (Sec. 3.3): the curve traced by a disk of radius rho
// rolled around the pair, i.e. both disks' outer arcs joined by two concave
// waist arcs of radius rho; nodes uniform in arc length at (p + 1/2) L / M_p
// counterclockwise from the upper tangent point on disk 1.
__host__ __device__ inline void peanut_node(const PairFrame& f, double rho, int p, int Mp,
                                            double* x, double* y) {
  const double d = f.d, r1 = f.r1, r2 = f.r2;
  const double R1 = r1 + rho, R2 = r2 + rho;
  const double wx = (d * d + R1 * R1 - R2 * R2) / (2.0 * d);
  const double wy = sqrt(fmax(R1 * R1 - wx * wx, 0.0));
  const double th1 = atan2(wy, wx), th2 = atan2(wy, wx - d);
  const double a1 = atan2(wy, -wx), a2 = atan2(wy, d - wx);
  // arcs: (centre x, centre y, radius, t0, t1)
  const double cx[4] = {0.0, wx, d, wx};
  const double cy[4] = {0.0, -wy, 0.0, wy};
  const double rr[4] = {r1, rho, r2, rho};
  const double t0[4] = {th1, a1, -th2, -a2};
  const double t1[4] = {2.0 * LMFS_PI - th1, a2, th2, -a1};
  double len[4], L = 0.0;
  for (int q = 0; q < 4; ++q) { len[q] = rr[q] * fabs(t1[q] - t0[q]); L += len[q]; }
  const double s = (p + 0.5) * L / Mp;
  double start = 0.0;
  int q = 0;
  for (; q < 3; ++q) {
    if (s < start + len[q]) break;
    start += len[q];
  }
  const double t = t0[q] + (t1[q] - t0[q]) * (s - start) / len[q];
  const double lx = cx[q] + rr[q] * cos(t), ly = cy[q] + rr[q] * sin(t);
  *x = f.c1x + f.cphi * lx - f.sphi * ly;
  *y = f.c1y + f.sphi * lx + f.cphi * ly;
}

}  // namespace lmfs
