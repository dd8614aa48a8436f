/*
 * FP64 CPU oracle of the interface analyses run on the density field:
 * the contact angle of a sessile droplet (Section 4.2) and the connected
 * vapour / liquid regions used to detect bubble departure (Section 4.3).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/ (and nothing in the product
 * path).  It shares no code with the CUDA library.
 *
 * Contact angle.  The interface is the level rho_mid = (rho_l + rho_g) / 2
 * (the level the paper's diagnostics use).  Every lattice link between two
 * horizontally or vertically adjacent nodes whose densities lie on opposite
 * sides of rho_mid gives one interface point, placed on the link by linear
 * interpolation.  Links with a node closer than skip_rows to the south wall
 * are left out (the wetting ghost layer distorts the first rows).  A circle
 * is fitted to the points by algebraic least squares (minimise
 * sum (x^2 + y^2 + D x + E y + F)^2, the normal equations solved by Gaussian
 * elimination; coordinates are taken relative to the points' mean), and the
 * angle inside the liquid follows from where the circle meets the wall line
 * y_w: cos(theta) = (y_w - y_c) / R.  With halfway bounce-back the wall sits
 * half a lattice spacing below row 0, y_w = -1/2.
 *
 * Components.  Nodes with rho < threshold (below = 1, vapour) or
 * rho > threshold (below = 0, liquid) are split into 4-connected components,
 * across the periodic seams of periodic axes.  A raster scan (x fastest)
 * starts a breadth-first flood fill at every node not yet labelled, so each
 * component's label is the smallest node index y * nx + x it contains.
 * Per component: node count, row range, contact with each edge, and the sum
 * of row indices.
 *
 * Pins (tests/test_oracle_analysis.py): the fit recovers exact circles to
 * round-off; caps built from tanh profiles around circles of known angle
 * give that angle; the components match scipy.ndimage.label on non-periodic
 * masks and hand-counted periodic cases.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* interface points on links (x,y)-(x+1,y) and (x,y)-(x,y+1) */
int orc_interface_points(const double* rho, int nx, int ny, double rho_mid, int skip_rows,
                         double* px, double* py, int max_points) {
    if (!rho || nx < 1 || ny < 1 || skip_rows < 0) return ORC_EINVAL;
    int n = 0;
    for (int y = skip_rows; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const double a = rho[(size_t)y * nx + x] - rho_mid;
            if (x + 1 < nx) {
                const double b = rho[(size_t)y * nx + x + 1] - rho_mid;
                if ((a >= 0.0) != (b >= 0.0)) {
                    if (n < max_points && px && py) {
                        px[n] = x + a / (a - b);
                        py[n] = y;
                    }
                    ++n;
                }
            }
            if (y + 1 < ny) {
                const double b = rho[(size_t)(y + 1) * nx + x] - rho_mid;
                if ((a >= 0.0) != (b >= 0.0)) {
                    if (n < max_points && px && py) {
                        px[n] = x;
                        py[n] = y + a / (a - b);
                    }
                    ++n;
                }
            }
        }
    return n;
}

/* Gaussian elimination with partial pivoting of a 3 x 3 system */
static int solve3(double A[3][3], double b[3], double x[3]) {
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return ORC_EINVAL;
        if (piv != c) {
            for (int k = 0; k < 3; ++k) {
                double t = A[c][k];
                A[c][k] = A[piv][k];
                A[piv][k] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < 3; ++r) {
            const double m = A[r][c] / A[c][c];
            for (int k = c; k < 3; ++k) A[r][k] -= m * A[c][k];
            b[r] -= m * b[c];
        }
    }
    for (int r = 2; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < 3; ++k) s -= A[r][k] * x[k];
        x[r] = s / A[r][r];
    }
    return ORC_OK;
}

int orc_circle_fit(const double* px, const double* py, int n, double out[3]) {
    if (!px || !py || !out || n < 3) return ORC_EINVAL;
    double xm = 0.0, ym = 0.0;
    for (int i = 0; i < n; ++i) {
        xm += px[i];
        ym += py[i];
    }
    xm /= n;
    ym /= n;
    /* normal equations of min sum (z + D u + E v + F)^2, z = u^2 + v^2 */
    double A[3][3] = {{0}}, b[3] = {0};
    for (int i = 0; i < n; ++i) {
        const double u = px[i] - xm, v = py[i] - ym, z = u * u + v * v;
        const double r[3] = {u, v, 1.0};
        for (int j = 0; j < 3; ++j) {
            for (int k = 0; k < 3; ++k) A[j][k] += r[j] * r[k];
            b[j] -= r[j] * z;
        }
    }
    double s[3];
    if (solve3(A, b, s)) return ORC_EINVAL;
    const double uc = -0.5 * s[0], vc = -0.5 * s[1];
    const double R2 = uc * uc + vc * vc - s[2];
    if (!(R2 > 0.0)) return ORC_EINVAL;
    out[0] = xm + uc;
    out[1] = ym + vc;
    out[2] = sqrt(R2);
    return ORC_OK;
}

int orc_contact_angle(const double* rho, int nx, int ny, double rho_l, double rho_g,
                      int skip_rows, orc_contact* out) {
    if (!rho || !out || !(rho_l > rho_g)) return ORC_EINVAL;
    memset(out, 0, sizeof(*out));
    const double rmid = 0.5 * (rho_l + rho_g);
    int n = orc_interface_points(rho, nx, ny, rmid, skip_rows, NULL, NULL, 0);
    if (n < 0) return n;
    out->n_points = n;
    if (n < 3) return ORC_EINVAL;
    double* px = (double*)malloc(sizeof(double) * n);
    double* py = (double*)malloc(sizeof(double) * n);
    if (!px || !py) {
        free(px);
        free(py);
        return ORC_ENOMEM;
    }
    orc_interface_points(rho, nx, ny, rmid, skip_rows, px, py, n);
    double c[3];
    int rc = orc_circle_fit(px, py, n, c);
    free(px);
    free(py);
    if (rc) return rc;
    const double yw = -0.5;
    out->xc = c[0];
    out->yc = c[1];
    out->radius = c[2];
    double cs = (yw - c[1]) / c[2];
    cs = cs < -1.0 ? -1.0 : (cs > 1.0 ? 1.0 : cs);
    out->theta_deg = acos(cs) * 180.0 / M_PI;
    const double h = c[2] * c[2] - (yw - c[1]) * (yw - c[1]);
    out->base_width = h > 0.0 ? 2.0 * sqrt(h) : 0.0;
    out->height = c[1] + c[2] - yw;
    return ORC_OK;
}

int orc_components(const double* rho, int nx, int ny, int periodic_x, int periodic_y,
                   double threshold, int below, int* labels, orc_component* comps,
                   int max_comps, int* n_comps) {
    if (!rho || !labels || nx < 1 || ny < 1 || !n_comps) return ORC_EINVAL;
    const size_t N = (size_t)nx * ny;
    int* queue = (int*)malloc(sizeof(int) * N);
    if (!queue) return ORC_ENOMEM;
    for (size_t i = 0; i < N; ++i) {
        const int in = below ? rho[i] < threshold : rho[i] > threshold;
        labels[i] = in ? -2 : -1;   /* -2: in the phase, not yet labelled */
    }
    int nc = 0;
    for (size_t s = 0; s < N; ++s) {
        if (labels[s] != -2) continue;
        /* flood fill from the first unlabelled node of the raster scan */
        const int lab = (int)s;
        size_t head = 0, tail = 0;
        queue[tail++] = lab;
        labels[s] = lab;
        orc_component c;
        memset(&c, 0, sizeof(c));
        c.label = lab;
        c.y_min = ny;
        c.y_max = -1;
        while (head < tail) {
            const int i = queue[head++];
            const int x = i % nx, y = i / nx;
            c.area += 1;
            c.sum_y += y;
            if (y < c.y_min) c.y_min = y;
            if (y > c.y_max) c.y_max = y;
            if (x == 0) c.touches_w = 1;
            if (x == nx - 1) c.touches_e = 1;
            if (y == 0) c.touches_s = 1;
            if (y == ny - 1) c.touches_n = 1;
            /* 4-neighbours, wrapped across periodic seams */
            int nb[4][2] = {{x - 1, y}, {x + 1, y}, {x, y - 1}, {x, y + 1}};
            for (int k = 0; k < 4; ++k) {
                int xx = nb[k][0], yy = nb[k][1];
                if (xx < 0 || xx >= nx) {
                    if (!periodic_x) continue;
                    xx = (xx + nx) % nx;
                }
                if (yy < 0 || yy >= ny) {
                    if (!periodic_y) continue;
                    yy = (yy + ny) % ny;
                }
                const size_t j = (size_t)yy * nx + xx;
                if (labels[j] == -2) {
                    labels[j] = lab;
                    queue[tail++] = (int)j;
                }
            }
        }
        if (nc < max_comps && comps) comps[nc] = c;
        ++nc;
    }
    free(queue);
    *n_comps = nc;
    return ORC_OK;
}
