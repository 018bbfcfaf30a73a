// FP64 build of the cell-interaction tensor N and of its reduced real spectrum (one-off, off the
// time-stepping path).  With P uniform in each cell (Sec. 3) and P = 0 outside the sample
// (Sec. 2), the cell-averaged field of Eq. 6 is E_el(a) = -(1/(eps0 epsB)) sum_b N(r_a - r_b) P(b)
// with N the cell-pair averaged demagnetization-type tensor the paper borrows from
// magnetostatics [40].
//
//  * near offsets: Newell-Williams-Dunlop closed forms (J. Geophys. Res. 98 (1993) 9551): the
//    27-point mixed second difference of f (diagonal) or g (off-diagonal) / (4 pi V);
//  * far offsets: -(V/4 pi) times the average of the point-dipole kernel (3 u u^T - |u|^2 I)/|u|^5
//    over the separation u = R + s of two uniform points, s distributed as the product of three
//    triangle densities on [-d_i, d_i]; each triangle half carries an m-point Gauss-Legendre rule.
//
// Spectrum: on the zero-padded grid (M_i >= 2 n_i - 1) the tensor is even (diagonal components)
// or odd (N_ij, i != j, odd along i and j) along each axis, so its DFT is real and is a separable
// sum of cosine and sine transforms; only kx <= Mx/2, ky <= My/2, kz <= Mz/2 is stored.
#pragma once
#include <cuda_runtime.h>

namespace tdgl {

// component order: xx yy zz xy xz yz
__device__ __constant__ int c_odd[6][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};

__device__ __forceinline__ double newell_fd(double x, double y, double z) {
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z, R = sqrt(xx + yy + zz);
    double v = (2.0 * xx - yy - zz) * R * (1.0 / 6.0);
    const double rxz = sqrt(xx + zz), rxy = sqrt(xx + yy);
    if (y > 0.0 && rxz > 0.0) v += 0.5 * y * (zz - xx) * asinh(y / rxz);
    if (z > 0.0 && rxy > 0.0) v += 0.5 * z * (yy - xx) * asinh(z / rxy);
    if (x > 0.0 && y > 0.0 && z > 0.0) v -= x * y * z * atan((y * z) / (x * R));
    return v;
}

__device__ __forceinline__ double newell_gd(double x, double y, double z) {
    const double sgn = (x < 0.0 ? -1.0 : 1.0) * (y < 0.0 ? -1.0 : 1.0);
    x = fabs(x); y = fabs(y); z = fabs(z);
    const double xx = x * x, yy = y * y, zz = z * z, R = sqrt(xx + yy + zz);
    double v = -x * y * R * (1.0 / 3.0);
    if (x > 0.0 && y > 0.0) {
        v += (y * (1.0 / 6.0)) * (3.0 * zz - yy) * asinh(x / sqrt(yy + zz));
        v += (x * (1.0 / 6.0)) * (3.0 * zz - xx) * asinh(y / sqrt(xx + zz));
        if (z > 0.0) {
            v += x * y * z * asinh(z / sqrt(xx + yy));
            v -= (zz * z * (1.0 / 6.0)) * atan((x * y) / (z * R));
            v -= 0.5 * z * yy * atan((x * z) / (y * R));
            v -= 0.5 * z * xx * atan((y * z) / (x * R));
        }
    }
    return sgn * v;
}

template <bool G>
__device__ double mixed_diff(double X, double Y, double Z, double a, double b, double c) {
    double s = 0.0;
    for (int i = -1; i <= 1; ++i) {
        const double wi = i ? -1.0 : 2.0;
        for (int j = -1; j <= 1; ++j) {
            const double wij = wi * (j ? -1.0 : 2.0);
            for (int k = -1; k <= 1; ++k) {
                const double w = wij * (k ? -1.0 : 2.0);
                const double u = X + i * a, v = Y + j * b, t = Z + k * c;
                s += w * (G ? newell_gd(u, v, t) : newell_fd(u, v, t));
            }
        }
    }
    return s;
}

// quadrature table: for each rule q (0..2), nq[q] points tau in (0,1) with weight
// (1 - tau) * w_GL / 2, mirrored to +-tau
struct FarRule {
    int m[3];
    double tau[3][8];
    double wt[3][8];
};

__global__ void k_tensor_real(double *__restrict__ out, int nx, int ny, int nz, double dx, double dy, double dz,
                              double r_newell, double r_q1, double r_q2, FarRule rule) {
    const long n = (long)nx * ny * nz;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < n; id += (long)gridDim.x * blockDim.x) {
        const int i = (int)(id % nx), j = (int)((id / nx) % ny), k = (int)(id / ((long)nx * ny));
        const double X = i * dx, Y = j * dy, Z = k * dz;
        const double dm = fmax(dx, fmax(dy, dz));
        const double r = sqrt(X * X + Y * Y + Z * Z) / dm;
        double v[6];
        if (r < r_newell) {
            const double s = 1.0 / (4.0 * 3.14159265358979323846 * dx * dy * dz);
            v[0] = s * mixed_diff<false>(X, Y, Z, dx, dy, dz);
            v[1] = s * mixed_diff<false>(Y, X, Z, dy, dx, dz);
            v[2] = s * mixed_diff<false>(Z, Y, X, dz, dy, dx);
            v[3] = s * mixed_diff<true>(X, Y, Z, dx, dy, dz);
            v[4] = s * mixed_diff<true>(X, Z, Y, dx, dz, dy);
            v[5] = s * mixed_diff<true>(Y, Z, X, dy, dz, dx);
        } else {
            const int q = (r < r_q1) ? 0 : ((r < r_q2) ? 1 : 2);
            const int m = rule.m[q];
            double acc[6] = {0, 0, 0, 0, 0, 0};
            for (int a = 0; a < 2 * m; ++a) {
                const double sa = (a & 1 ? -1.0 : 1.0) * rule.tau[q][a >> 1], wa = rule.wt[q][a >> 1];
                const double ux = X + sa * dx;
                for (int b = 0; b < 2 * m; ++b) {
                    const double sb = (b & 1 ? -1.0 : 1.0) * rule.tau[q][b >> 1], wb = wa * rule.wt[q][b >> 1];
                    const double uy = Y + sb * dy;
                    for (int c = 0; c < 2 * m; ++c) {
                        const double sc = (c & 1 ? -1.0 : 1.0) * rule.tau[q][c >> 1], w = wb * rule.wt[q][c >> 1];
                        const double uz = Z + sc * dz;
                        const double u2 = ux * ux + uy * uy + uz * uz;
                        const double iu = rsqrt(u2);
                        const double i5 = w * iu * iu * iu / u2;   // w / |u|^5
                        acc[0] += (3.0 * ux * ux - u2) * i5;
                        acc[1] += (3.0 * uy * uy - u2) * i5;
                        acc[2] += (3.0 * uz * uz - u2) * i5;
                        acc[3] += 3.0 * ux * uy * i5;
                        acc[4] += 3.0 * ux * uz * i5;
                        acc[5] += 3.0 * uy * uz * i5;
                    }
                }
            }
            const double s = -dx * dy * dz / (4.0 * 3.14159265358979323846);
            for (int c = 0; c < 6; ++c) v[c] = s * acc[c];
        }
        for (int c = 0; c < 6; ++c) out[c * n + id] = v[c];
    }
}

// One separable pass along axis `ax` (0 = x fastest, 1 = y, 2 = z) of the reduced transform:
//   out[c][..k..] = sum_{o=0}^{n-1} w_c(o) in[c][..o..] trig_c(k o mod M)
// even along ax: w = 1 (o = 0), 2 (o > 0), trig = cos;  odd: w = 0 (o = 0), 2, trig = sin.
// in has extent n along ax, out has extent K = M/2 + 1; the other two extents e0 (inner),
// e1 (outer) are shared.  The (-i) factor of each odd axis is applied by the last pass.
__global__ void k_tensor_dft(const double *__restrict__ in, double *__restrict__ out, int ax, int n, int K,
                             int M, int inner, int outer, const double *__restrict__ cs, const double *__restrict__ sn) {
    // in layout [6][outer][n][inner]; out layout [6][outer][K][inner]
    const long per = (long)outer * K * inner;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < 6 * per; id += (long)gridDim.x * blockDim.x) {
        const int c = (int)(id / per);
        const long r = id - c * per;
        const int i0 = (int)(r % inner);
        const int k = (int)((r / inner) % K);
        const int o1 = (int)(r / ((long)inner * K));
        const bool odd = c_odd[c][ax] != 0;
        const double *src = in + ((long)c * outer + o1) * (long)n * inner + i0;
        double s = 0.0;
        int t = 0;   // k*o mod M
        for (int o = 0; o < n; ++o) {
            const double val = src[(long)o * inner];
            if (odd) s += (o ? 2.0 : 0.0) * val * sn[t];
            else s += (o ? 2.0 : 1.0) * val * cs[t];
            t += k;
            if (t >= M) t -= M;
        }
        out[id] = s;
    }
}

// final conversion to the float table the convolution reads: sign (-i)^(number of odd axes)
// -> -1 for the off-diagonal components; components paired as float2 planes (xx, yy), (zz, xy),
// (xz, yz), rows of kxp entries (kxp >= Kx, the row pitch of the spectra, padding zero).
// in: [6][rows][Kx] float64; out: [3][rows][kxp] float2
__global__ void k_tensor_store(const double *__restrict__ in, float2 *__restrict__ out, long rows, int Kx, int kxp) {
    const long per = rows * kxp, per_in = rows * Kx;
    for (long id = blockIdx.x * (long)blockDim.x + threadIdx.x; id < 3 * per; id += (long)gridDim.x * blockDim.x) {
        const int j = (int)(id / per);
        const long rk = id - j * per, r = rk / kxp;
        const int kx = (int)(rk - r * kxp);
        float2 v = make_float2(0.f, 0.f);
        if (kx < Kx) {
            const long a = (2 * j) * per_in + r * Kx + kx, b = a + per_in;
            v.x = (float)((2 * j >= 3 ? -1.0 : 1.0) * in[a]);
            v.y = (float)((2 * j + 1 >= 3 ? -1.0 : 1.0) * in[b]);
        }
        out[id] = v;
    }
}

}  // namespace tdgl
