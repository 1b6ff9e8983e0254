// Host FP64 numerics of libqp: the short-time propagator U = exp(-i H_S dt)
// and the influence coefficients eta_d from a spectral density.
//
// eta_d (paper Eq. inf_fun; explicit forms deferred by the paper to its
// refs) is computed as the double integral of the bath correlation function
// alpha(t) = (1/pi) int_0^inf J(w)[coth(beta w/2) cos wt - i sin wt] dw over
// a pair of boxes of width dt that are d steps apart (the point q_k holds on
// ((k-1) dt, k dt]).  Doing the two time integrals analytically gives
//   eta_0 = (1/pi) int J/w^2 [coth(beta w/2)(1 - cos w dt) - i (w dt - sin w dt)] dw
//   eta_d = (4/pi) int J/w^2 sin^2(w dt/2) [coth(beta w/2) cos(w d dt) - i sin(w d dt)] dw,
// evaluated by adaptive composite Gauss-Legendre quadrature (20 vs 40 nodes
// per panel, nodes from Newton iteration on the Legendre recurrence).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace qp {

// ------------------------------------------------------------------ propagator

static void matmul(int M, const cplx *A, const cplx *B, cplx *C) {
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < M; ++k) s += A[i * M + k] * B[k * M + j];
            C[i * M + j] = s;
        }
}

void short_time_propagator(int M, const cplx *H, double dt, cplx *U) {
    // M <= 8: fixed arrays, no allocation (the allocation-free step uses it)
    // A = -i H dt, scaled by 2^-s so that its 1-norm is below 1/4
    cplx A[64], T[64], P[64], tmp[64];
    double norm = 0.0;
    for (int j = 0; j < M; ++j) {
        double col = 0.0;
        for (int i = 0; i < M; ++i) col += std::abs(H[i * M + j]) * std::fabs(dt);
        norm = std::max(norm, col);
    }
    int s = 0;
    while (norm > 0.25) { norm *= 0.5; ++s; }
    const double scale = std::ldexp(1.0, -s);
    for (int i = 0; i < M * M; ++i) A[i] = cplx(0.0, -1.0) * H[i] * dt * scale;
    // Taylor series to order 20: |A| < 1/4 gives a remainder far below 1e-17
    for (int i = 0; i < M * M; ++i) { T[i] = 0.0; P[i] = 0.0; }
    for (int i = 0; i < M; ++i) { T[i * M + i] = 1.0; P[i * M + i] = 1.0; }
    for (int k = 1; k <= 20; ++k) {
        matmul(M, P, A, tmp);
        for (int i = 0; i < M * M; ++i) { P[i] = tmp[i] / double(k); T[i] += P[i]; }
    }
    for (int r = 0; r < s; ++r) {
        matmul(M, T, T, tmp);
        for (int i = 0; i < M * M; ++i) T[i] = tmp[i];
    }
    for (int i = 0; i < M * M; ++i) U[i] = T[i];
}

std::vector<cplx> short_time_propagator(int M, const std::vector<cplx> &H, double dt) {
    std::vector<cplx> U(M * M);
    short_time_propagator(M, H.data(), dt, U.data());
    return U;
}

// ------------------------------------------------------------------ bath

double spectral_density(const qp_bath &b, double w) {
    double j = 0.0;
    if (b.ohmic_alpha != 0.0) j += 0.5 * M_PI * b.ohmic_alpha * w * std::exp(-w / b.ohmic_wc);
    if (b.res_lambda != 0.0) {
        // Eq. sharpSD: J = 2 a w W^4 / ((W^2 - w^2)^2 + (g w)^2), with
        // lambda = int J/w dw = pi a W^2 / g fixing the amplitude a
        const double W = b.res_w0, g = b.res_gamma;
        const double a = b.res_lambda * g / (M_PI * W * W);
        const double d = W * W - w * w;
        j += 2.0 * a * w * W * W * W * W / (d * d + g * g * w * w);
    }
    return j;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double pp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int k = 1; k <= n; ++k) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * k - 1.0) * z * p2 - (k - 1.0) * p3) / k;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

namespace {

struct EtaIntegrand {
    const qp_bath *b;
    double dt;
    int n;
    // out[2*d] = Re, out[2*d+1] = Im integrand of eta_d at frequency w (times pi)
    void operator()(double w, double *out) const {
        const double jw = spectral_density(*b, w) / (w * w);
        const double coth = 1.0 / std::tanh(0.5 * b->beta * w);
        const double x = w * dt;
        const double sh = std::sin(0.5 * x);
        // eta_0: coth(1 - cos x) - i (x - sin x)
        double xms;
        if (x < 0.1) {
            const double x2 = x * x;
            xms = x * x2 / 6.0 * (1 - x2 / 20.0 * (1 - x2 / 42.0 * (1 - x2 / 72.0 * (1 - x2 / 110.0))));
        } else {
            xms = x - std::sin(x);
        }
        out[0] = jw * coth * 2.0 * sh * sh;
        out[1] = -jw * xms;
        const double box = 4.0 * jw * sh * sh;
        for (int d = 1; d < n; ++d) {
            const double ph = x * d;
            out[2 * d] = box * coth * std::cos(ph);
            out[2 * d + 1] = -box * std::sin(ph);
        }
    }
};

// Q(t) = (1/pi) int J(w)/w^2 [coth(beta w/2)(1 - cos wt) - i (wt - sin wt)] dw
// at t = j h, j = 0 .. n-1 (times pi): the double integral of the bath
// correlation function from 0, whose second differences are the influence
// coefficients of full intervals.
struct QIntegrand {
    const qp_bath *b;
    double h;
    int n;
    void operator()(double w, double *out) const {
        const double jw = spectral_density(*b, w) / (w * w);
        const double coth = 1.0 / std::tanh(0.5 * b->beta * w);
        for (int j = 0; j < n; ++j) {
            const double x = w * h * j;
            double xms;
            if (x < 0.1) {
                const double x2 = x * x;
                xms = x * x2 / 6.0 * (1 - x2 / 20.0 * (1 - x2 / 42.0 * (1 - x2 / 72.0 * (1 - x2 / 110.0))));
            } else {
                xms = x - std::sin(x);
            }
            const double sh = std::sin(0.5 * x);
            out[2 * j] = jw * coth * 2.0 * sh * sh;
            out[2 * j + 1] = -jw * xms;
        }
    }
};

struct Quad {
    std::vector<double> x20, w20, x40, w40;
    Quad() {
        gauss_legendre(20, x20, w20);
        gauss_legendre(40, x40, w40);
    }
};

template <typename F>
void panel(const F &f, const Quad &Q, double a, double b, int nout,
           std::vector<double> &r20, std::vector<double> &r40, std::vector<double> &buf) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    std::fill(r20.begin(), r20.end(), 0.0);
    std::fill(r40.begin(), r40.end(), 0.0);
    for (int i = 0; i < 20; ++i) {
        f(c + h * Q.x20[i], buf.data());
        for (int k = 0; k < nout; ++k) r20[k] += h * Q.w20[i] * buf[k];
    }
    for (int i = 0; i < 40; ++i) {
        f(c + h * Q.x40[i], buf.data());
        for (int k = 0; k < nout; ++k) r40[k] += h * Q.w40[i] * buf[k];
    }
}

}  // namespace

// Adaptive Gauss-Legendre (20/40 points) of nout integrands over frequency,
// split at the bath's scales; panels no wider than hmax.  acc gets the sums.
template <typename F>
void integrate_bath(const qp_bath &b, const F &f, int nout, double hmax, std::vector<double> &acc) {
    const Quad Q;
    // breakpoints: ohmic scale and the resonance peak; oscillation period of
    // the largest lag bounds the panel width
    std::vector<double> pts{0.0};
    double wmax = 0.0;
    if (b.ohmic_alpha != 0.0) {
        for (double m : {0.5, 1.0, 2.0, 5.0, 10.0, 20.0, 40.0}) pts.push_back(m * b.ohmic_wc);
        wmax = std::max(wmax, 60.0 * b.ohmic_wc);
    }
    if (b.res_lambda != 0.0) {
        for (double k : {0.0, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0}) {
            pts.push_back(b.res_w0 - k * b.res_gamma);
            pts.push_back(b.res_w0 + k * b.res_gamma);
        }
        wmax = std::max(wmax, 4000.0 * std::max(1.0, b.res_w0));
    }
    pts.push_back(wmax);
    std::sort(pts.begin(), pts.end());
    pts.erase(std::remove_if(pts.begin(), pts.end(), [&](double p) { return p < 0.0 || p > wmax; }), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    acc.assign(nout, 0.0);
    std::vector<double> r20(nout), r40(nout), buf(nout);
    struct Seg { double a, b; int depth; };
    std::vector<Seg> stack;
    for (size_t i = 0; i + 1 < pts.size(); ++i) {
        const double a = pts[i], bb = pts[i + 1];
        const int np = std::max(1, int(std::ceil((bb - a) / hmax)));
        for (int k = np - 1; k >= 0; --k) stack.push_back({a + (bb - a) * k / np, a + (bb - a) * (k + 1) / np, 0});
        while (!stack.empty()) {
            Seg s = stack.back();
            stack.pop_back();
            panel(f, Q, s.a, s.b, nout, r20, r40, buf);
            double err = 0.0;
            for (int k = 0; k < nout; ++k) err = std::max(err, std::fabs(r40[k] - r20[k]));
            if (err > 1e-17 && s.depth < 40) {
                const double m = 0.5 * (s.a + s.b);
                stack.push_back({m, s.b, s.depth + 1});
                stack.push_back({s.a, m, s.depth + 1});
            } else {
                for (int k = 0; k < nout; ++k) acc[k] += r40[k];
            }
        }
    }
}

static bool bath_ok(const qp_bath &b) {
    if (!(b.beta > 0.0)) return false;
    if (b.ohmic_alpha != 0.0 && !(b.ohmic_wc > 0.0)) return false;
    if (b.res_lambda != 0.0 && (!(b.res_w0 > 0.0) || !(b.res_gamma > 0.0) || b.res_gamma >= 2.0 * b.res_w0))
        return false;
    return true;
}

int eta_from_bath(const qp_bath &b, double dt, int n, std::vector<cplx> &eta) {
    if (!bath_ok(b) || !(dt > 0.0) || n < 1) return 1;
    EtaIntegrand f{&b, dt, n};
    std::vector<double> acc;
    integrate_bath(b, f, 2 * n, std::max(1e-3, 1.0 / (dt * std::max(1, n))), acc);
    eta.assign(n, cplx(0.0, 0.0));
    for (int d = 0; d < n; ++d) eta[d] = cplx(acc[2 * d], acc[2 * d + 1]) / M_PI;
    return 0;
}

int Q_from_bath(const qp_bath &b, double h, int n, std::vector<cplx> &Q) {
    if (!bath_ok(b) || !(h > 0.0) || n < 1) return 1;
    QIntegrand f{&b, h, n};
    std::vector<double> acc;
    integrate_bath(b, f, 2 * n, std::max(1e-3, 1.0 / (h * std::max(1, n))), acc);
    Q.assign(n, cplx(0.0, 0.0));
    for (int j = 0; j < n; ++j) Q[j] = cplx(acc[2 * j], acc[2 * j + 1]) / M_PI;
    return 0;
}

}  // namespace qp
