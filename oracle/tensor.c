/*
 * ORACLE (test infrastructure only; never part of the product path).
 *
 * FP64 cell-interaction tensor N for the open-boundary electrostatic field of Eqs. 5-6:
 *   E_el(cell a) = -(1/(eps0 epsB)) * sum_b N(r_a - r_b) P(b),
 * where N is the cell-pair average of the field of a uniformly polarized cuboid cell over
 * another cell of the same shape (Sec. 2: P uniform in each cell; the paper computes this
 * field "similar to magnetostatics" [40], i.e. with the magnetostatic demagnetization tensor).
 *
 * Two independent evaluations:
 *  - near field: the closed forms of Newell, Williams and Dunlop (J. Geophys. Res. 98, 9551,
 *    1993): N_xx is the 27-point second mixed difference of their function f, N_xy that of g,
 *    divided by 4 pi dx dy dz.  Exact, but the differences cancel catastrophically with distance.
 *  - far field: the same cell-pair average written as an integral of the point-dipole kernel
 *    against the tent (triangle) density of the separation of two uniform points of two
 *    cells, evaluated with a tensor-product Gauss-Legendre rule on each half of the tent.
 * The tests check both against each other on an overlap band, and against closed forms.
 *
 * Component order everywhere: xx, yy, zz, xy, xz, yz.
 */
#include <math.h>
#include <stdlib.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Newell f(x,y,z); even in every argument. */
static double newell_f(double x, double y, double z)
{
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    double r = 0.0;
    if (y > 0.0 && (z2 - x2) != 0.0) {
        double d = sqrt(x2 + z2);
        if (d > 0.0) r += 0.5 * y * (z2 - x2) * asinh(y / d);
    }
    if (z > 0.0 && (y2 - x2) != 0.0) {
        double d = sqrt(x2 + y2);
        if (d > 0.0) r += 0.5 * z * (y2 - x2) * asinh(z / d);
    }
    if (x > 0.0 && y > 0.0 && z > 0.0) r -= x * y * z * atan(y * z / (x * R));
    r += (2.0 * x2 - y2 - z2) * R / 6.0;
    return r;
}

/* Newell g(x,y,z); odd in x and in y, even in z. */
static double newell_g(double x, double y, double z)
{
    double s = ((x < 0.0) ? -1.0 : 1.0) * ((y < 0.0) ? -1.0 : 1.0);
    x = fabs(x); y = fabs(y); z = fabs(z);
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double R = sqrt(x2 + y2 + z2);
    double r = 0.0;
    if (x > 0.0 && y > 0.0 && z > 0.0) r += x * y * z * asinh(z / sqrt(x2 + y2));
    if (y > 0.0 && x > 0.0) r += y / 6.0 * (3.0 * z2 - y2) * asinh(x / sqrt(y2 + z2));
    if (x > 0.0 && y > 0.0) r += x / 6.0 * (3.0 * z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (z > 0.0 && x > 0.0 && y > 0.0) r -= z2 * z / 6.0 * atan(x * y / (z * R));
    if (z > 0.0 && y > 0.0 && x > 0.0) r -= 0.5 * z * y2 * atan(x * z / (y * R));
    if (z > 0.0 && x > 0.0 && y > 0.0) r -= 0.5 * z * x2 * atan(y * z / (x * R));
    r -= x * y * R / 3.0;
    return s * r;
}

/* 27-point mixed difference, weights 2 (centre) / -1 (either side) per axis. */
static double diff27(double (*fn)(double, double, double), double X, double Y, double Z,
                     double a, double b, double c)
{
    static const double w[3] = {-1.0, 2.0, -1.0};
    double s = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k)
                s += w[i] * w[j] * w[k] * fn(X + (i - 1) * a, Y + (j - 1) * b, Z + (k - 1) * c);
    return s;
}

/* Near-field tensor at offset (X,Y,Z) (metres) for cells dx x dy x dz. */
void oracle_tensor_newell(double X, double Y, double Z, double dx, double dy, double dz,
                          double out[6])
{
    double s = 1.0 / (4.0 * M_PI * dx * dy * dz);
    out[0] = s * diff27(newell_f, X, Y, Z, dx, dy, dz);
    out[1] = s * diff27(newell_f, Y, X, Z, dy, dx, dz);
    out[2] = s * diff27(newell_f, Z, Y, X, dz, dy, dx);
    out[3] = s * diff27(newell_g, X, Y, Z, dx, dy, dz);
    out[4] = s * diff27(newell_g, X, Z, Y, dx, dz, dy);
    out[5] = s * diff27(newell_g, Y, Z, X, dy, dz, dx);
}

/* Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_m. */
static void gauss_legendre(int m, double *t, double *w)
{
    for (int i = 0; i < m; ++i) {
        double x = cos(M_PI * (i + 0.75) / (m + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= m; ++k) {
                double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double dp = m * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double p0 = 1.0, p1 = x;
        for (int k = 2; k <= m; ++k) {
            double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1; p1 = p2;
        }
        double dp = m * (x * p1 - p0) / (x * x - 1.0);
        t[i] = x;
        w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

#define MAXQ 64
/* Far-field tensor: -(V/4pi) * int tent(s) (3 u u^T/|u|^2 - I)/|u|^3, u = R + s.
 * Each axis: int_{-D}^{D} (1-|s|/D)/D phi(s) ds = int_0^1 (1-t) [phi(Dt) + phi(-Dt)] dt,
 * integrated with m Gauss-Legendre points on [0,1]. */
void oracle_tensor_far(double X, double Y, double Z, double dx, double dy, double dz, int m,
                       double out[6])
{
    double t[MAXQ], w[MAXQ];
    double sx[2 * MAXQ], sy[2 * MAXQ], sz[2 * MAXQ], q[2 * MAXQ];
    if (m > MAXQ) m = MAXQ;
    gauss_legendre(m, t, w);
    int n = 0;
    for (int i = 0; i < m; ++i) {
        double tau = 0.5 * (1.0 + t[i]);
        double wt = 0.5 * w[i] * (1.0 - tau);
        sx[n] = dx * tau; sy[n] = dy * tau; sz[n] = dz * tau; q[n] = wt; ++n;
        sx[n] = -dx * tau; sy[n] = -dy * tau; sz[n] = -dz * tau; q[n] = wt; ++n;
    }
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double ux = X + sx[i], uy = Y + sy[j], uz = Z + sz[k];
                double r2 = ux * ux + uy * uy + uz * uz;
                double r = sqrt(r2);
                double ir5 = 1.0 / (r2 * r2 * r);
                double wq = q[i] * q[j] * q[k];
                acc[0] += wq * (3.0 * ux * ux - r2) * ir5;
                acc[1] += wq * (3.0 * uy * uy - r2) * ir5;
                acc[2] += wq * (3.0 * uz * uz - r2) * ir5;
                acc[3] += wq * 3.0 * ux * uy * ir5;
                acc[4] += wq * 3.0 * ux * uz * ir5;
                acc[5] += wq * 3.0 * uy * uz * ir5;
            }
    double s = -dx * dy * dz / (4.0 * M_PI);
    for (int c = 0; c < 6; ++c) out[c] = s * acc[c];
}

/* Tensor at integer cell offset (i,j,k).  Switch (distances in units of the largest cell edge,
 * chosen by comparing both methods with an extended-precision Newell evaluation):
 *   r < 4        Newell closed forms (FP64 cancellation error below ~1e-11 there),
 *   4 <= r < 16  far-field rule with 8 points per tent half,
 *   16 <= r < 48 6 points, r >= 48 4 points (rule error far below 1e-13 in both). */
void oracle_tensor_offset(int i, int j, int k, double dx, double dy, double dz, double out[6])
{
    double X = i * dx, Y = j * dy, Z = k * dz;
    double dm = dx > dy ? dx : dy;
    if (dz > dm) dm = dz;
    double rr = sqrt(X * X + Y * Y + Z * Z) / dm;
    if (rr < 4.0)
        oracle_tensor_newell(X, Y, Z, dx, dy, dz, out);
    else
        oracle_tensor_far(X, Y, Z, dx, dy, dz, rr < 16.0 ? 8 : (rr < 48.0 ? 6 : 4), out);
}

/* All offsets of one octant: out[c][k][j][i] for i in [0,nx), j in [0,ny), k in [0,nz). */
void oracle_tensor_octant(int nx, int ny, int nz, double dx, double dy, double dz, double *out)
{
    long plane = (long)nx * ny * nz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double v[6];
                oracle_tensor_offset(i, j, k, dx, dy, dz, v);
                long idx = ((long)k * ny + j) * nx + i;
                for (int c = 0; c < 6; ++c) out[c * plane + idx] = v[c];
            }
}
