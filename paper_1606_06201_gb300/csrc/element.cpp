// Element stiffness matrices (Sec. 7: square Q1 elements, isotropic E, nu; plane stress in 2D,
// the trilinear hexahedron in 3D) by tensor Gauss-Legendre quadrature with two points per
// direction, which integrates the bilinear / trilinear integrand exactly.
#include <cmath>
#include <cstring>

namespace topo {

namespace {

void gauss2(double* pts, double* wts) {
  const double g = 0.5 / std::sqrt(3.0);
  pts[0] = 0.5 - g;
  pts[1] = 0.5 + g;
  wts[0] = wts[1] = 0.5;
}

}  // namespace

// K0 for the unit square (2D, unit thickness) or unit cube (3D); row-major, local DOF order
// node-major (DOF = dim * local_node + component).
void element_stiffness_host(int dim, double E, double nu, double* K0) {
  double pts[2], wts[2];
  gauss2(pts, wts);
  if (dim == 2) {
    const double c = E / (1.0 - nu * nu);
    const double D[3][3] = {{c, c * nu, 0.0}, {c * nu, c, 0.0}, {0.0, 0.0, c * 0.5 * (1.0 - nu)}};
    const int cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
    std::memset(K0, 0, sizeof(double) * 64);
    for (int ga = 0; ga < 2; ++ga)
      for (int gb = 0; gb < 2; ++gb) {
        const double s = pts[ga], t = pts[gb], w = wts[ga] * wts[gb];
        double B[3][8] = {};
        for (int a = 0; a < 4; ++a) {
          const double fx = cx[a] ? s : 1.0 - s, fy = cy[a] ? t : 1.0 - t;
          const double dNx = (cx[a] ? 1.0 : -1.0) * fy, dNy = (cy[a] ? 1.0 : -1.0) * fx;
          B[0][2 * a] = dNx;
          B[1][2 * a + 1] = dNy;
          B[2][2 * a] = dNy;
          B[2][2 * a + 1] = dNx;
        }
        for (int i = 0; i < 8; ++i)
          for (int j = 0; j < 8; ++j) {
            double acc = 0.0;
            for (int p = 0; p < 3; ++p)
              for (int q = 0; q < 3; ++q) acc += B[p][i] * D[p][q] * B[q][j];
            K0[i * 8 + j] += w * acc;
          }
      }
    return;
  }
  const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = E / (2.0 * (1.0 + nu));
  double D[6][6] = {};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) D[i][j] = lam + (i == j ? 2.0 * mu : 0.0);
  D[3][3] = D[4][4] = D[5][5] = mu;
  const int cx[8] = {0, 1, 1, 0, 0, 1, 1, 0}, cy[8] = {0, 0, 1, 1, 0, 0, 1, 1};
  const int cz[8] = {0, 0, 0, 0, 1, 1, 1, 1};
  std::memset(K0, 0, sizeof(double) * 576);
  for (int ga = 0; ga < 2; ++ga)
    for (int gb = 0; gb < 2; ++gb)
      for (int gc = 0; gc < 2; ++gc) {
        const double s = pts[ga], t = pts[gb], r = pts[gc], w = wts[ga] * wts[gb] * wts[gc];
        double B[6][24] = {};
        for (int a = 0; a < 8; ++a) {
          const double fx = cx[a] ? s : 1.0 - s, fy = cy[a] ? t : 1.0 - t, fz = cz[a] ? r : 1.0 - r;
          const double sx = cx[a] ? 1.0 : -1.0, sy = cy[a] ? 1.0 : -1.0, sz = cz[a] ? 1.0 : -1.0;
          const double dx = sx * fy * fz, dy = sy * fx * fz, dz = sz * fx * fy;
          B[0][3 * a] = dx;
          B[1][3 * a + 1] = dy;
          B[2][3 * a + 2] = dz;
          B[3][3 * a + 1] = dz;
          B[3][3 * a + 2] = dy;
          B[4][3 * a] = dz;
          B[4][3 * a + 2] = dx;
          B[5][3 * a] = dy;
          B[5][3 * a + 1] = dx;
        }
        for (int i = 0; i < 24; ++i)
          for (int j = 0; j < 24; ++j) {
            double acc = 0.0;
            for (int p = 0; p < 6; ++p)
              for (int q = 0; q < 6; ++q) acc += B[p][i] * D[p][q] * B[q][j];
            K0[i * 24 + j] += w * acc;
          }
      }
}

}  // namespace topo
