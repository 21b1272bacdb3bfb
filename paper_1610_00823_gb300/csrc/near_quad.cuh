// Quadrature of the log kernel and its gradient against the leaf basis over one
// source box, for the near-field tables of Section 3.1 (computed once for a unit box, reused at
// every level after scaling) and the gradient tables of Section 3.2.
//
// Target x (unit target box [-1/2, 1/2]^2 coordinates), source box S of centre c
// and width rho. p = the point of the closed box S nearest to x (p = x when x is
// inside). S is the union of the four triangles (p, P0, P1) over its edges, each
// mapped from (s, t) in [0, 1]^2 by y = p + s (P0 + t (P1 - P0) - p), Jacobian s D,
// D = cross(P0 - p, P1 - P0) >= 0 (triangles through p are skipped). Both s and
// t use the tanh-sinh (double exponential) rule, whose nodes crowd doubly
// exponentially at the ends of [0, 1]: the kernel singularity sits at s = 0 (x
// inside, or x at distance |x - p| outside), and the near-singularity in t at
// the foot t0 of the perpendicular from p is moved to an end by splitting
// [0, 1] at t0.
//
// Basis: Lagrange polynomials on the k first-kind Chebyshev nodes of the unit
// interval, evaluated by the barycentric formula with weights
// (-1)^j sin((2j + 1) pi / (2k)).
#pragma once

#include <cmath>

namespace vfmm {

struct DENode {
    double x, xc, w;  // node in (0, 1), 1 - node, weight
};

// Node j in [-n, n] of the tanh-sinh rule with step h on [0, 1]:
// x = 1 / (1 + exp(-pi sinh u)), u = j h, weight h pi cosh(u) x (1 - x).
__host__ __device__ inline DENode de_node(int j, double h) {
    const double pi = 3.14159265358979323846;
    double u = j * h;
    double e = exp(-pi * sinh(u));
    DENode d;
    d.x = 1.0 / (1.0 + e);
    d.xc = e / (1.0 + e);
    d.w = h * pi * cosh(u) * d.x * d.xc;
    return d;
}

// Lagrange basis values at xn (unit-interval coordinates) into out[k].
__host__ __device__ inline void bary_basis(int k, const double* nodes, const double* bw, double xn, double* out) {
    double den = 0.0;
    int hit = -1;
    for (int j = 0; j < k; ++j) {
        double d = xn - nodes[j];
        if (d == 0.0) {
            hit = j;
            break;
        }
        out[j] = bw[j] / d;
        den += out[j];
    }
    if (hit >= 0) {
        for (int j = 0; j < k; ++j) out[j] = (j == hit) ? 1.0 : 0.0;
        return;
    }
    double inv = 1.0 / den;
    for (int j = 0; j < k; ++j) out[j] *= inv;
}

struct QuadPiece {
    double px, py;    // apex
    double ax, ay;    // edge start P0
    double ex, ey;    // edge vector P1 - P0
    double D;         // cross(P0 - p, P1 - P0)
    double t0, t1;    // t sub-interval; the near-singular end is t0 when flip == 0
    int flip;         // 1: sigma measured from t1 downward
    int inside;       // x == p
};

// Up to 8 pieces (4 triangles x 2 halves in t).
__host__ __device__ inline int make_pieces(double x, double y, double cx, double cy, double rho, QuadPiece* pc) {
    const double hw = rho / 2.0;
    double lo_x = cx - hw, hi_x = cx + hw, lo_y = cy - hw, hi_y = cy + hw;
    double px = x < lo_x ? lo_x : (x > hi_x ? hi_x : x);
    double py = y < lo_y ? lo_y : (y > hi_y ? hi_y : y);
    int inside = (px == x && py == y);
    const double C[4][2] = {{lo_x, lo_y}, {hi_x, lo_y}, {hi_x, hi_y}, {lo_x, hi_y}};
    int n = 0;
    for (int e = 0; e < 4; ++e) {
        double ax = C[e][0], ay = C[e][1];
        double ex = C[(e + 1) % 4][0] - ax, ey = C[(e + 1) % 4][1] - ay;
        double D = (ax - px) * ey - (ay - py) * ex;
        if (!(D > 1e-300)) continue;
        double L2 = ex * ex + ey * ey;
        double tf = ((px - ax) * ex + (py - ay) * ey) / L2;
        tf = tf < 0.0 ? 0.0 : (tf > 1.0 ? 1.0 : tf);
        QuadPiece q{px, py, ax, ay, ex, ey, D, 0.0, 1.0, 0, inside};
        if (tf > 0.0) {
            q.t0 = 0.0;
            q.t1 = tf;
            q.flip = 1;
            pc[n++] = q;
        }
        if (tf < 1.0) {
            q.t0 = tf;
            q.t1 = 1.0;
            q.flip = 0;
            pc[n++] = q;
        }
    }
    return n;
}

// Weights of one quadrature node (piece, s-node, t-node): potential, d/dx1, d/dx2,
// and the node position y. Includes the -1/(2 pi) factor and the Jacobian.
__host__ __device__ inline void node_weights(const QuadPiece& q, double x, double y, const DENode& ds,
                                             const DENode& dt, double* w3, double* yx, double* yy) {
    const double inv2pi = 0.15915494309189533577;
    double len = q.t1 - q.t0;
    // t measured from the near-singular end
    double t = q.flip ? q.t1 - len * dt.x : q.t0 + len * dt.x;
    double wt = len * dt.w;
    double exx = q.ax + t * q.ex, eyy = q.ay + t * q.ey;  // edge point e(t)
    double vx = exx - q.px, vy = eyy - q.py;              // e(t) - p
    double s = ds.x;
    *yx = q.px + s * vx;
    *yy = q.py + s * vy;
    double J = q.D * wt * ds.w;  // D ds dt, times s below
    if (q.inside) {
        double r2 = vx * vx + vy * vy;
        double lr = 0.5 * log(r2);
        w3[0] = -inv2pi * J * s * (log(s) + lr);
        // (x - y)/|x - y|^2 * s = -(e - p)/r^2
        w3[1] = inv2pi * J * vx / r2;
        w3[2] = inv2pi * J * vy / r2;
    } else {
        double rx = x - *yx, ry = y - *yy;
        double rr = rx * rx + ry * ry;
        w3[0] = -inv2pi * J * s * 0.5 * log(rr);
        w3[1] = -inv2pi * J * s * rx / rr;
        w3[2] = -inv2pi * J * s * ry / rr;
    }
}

}  // namespace vfmm
