// circuit.cpp -- parameterised circuit -> Bargmann triple (A, b, c) with its
// Jacobian (host).  The circuit: M squeezed vacua (squeezing r_j of the x
// quadrature), real displacements x_j, an interferometer made of a triangle
// of M(M-1)/2 beam splitters on neighbouring modes and M output phases, and
// per-mode pure loss eta.  Parameters (M^2 + 2M of them):
//   [r_0..r_{M-1}, x_0..x_{M-1}, (theta_1, phi_1) .. (theta_nbs, phi_nbs),
//    psi_0..psi_{M-1}]
// with beam splitter (theta, phi) on modes (k, k+1) acting as
// [[cos t, -e^{-i phi} sin t], [e^{i phi} sin t, cos t]], applied in the
// order k = 0..M-2-i for i = 0..M-2, then the phases e^{i psi_j}.
//
// The triple follows Sec. 2.1, eqs. (A_rho), (b_rho) and the vacuum amplitude
// of Sec. 2.2 as in fk_gaussian_to_triple.  Its derivative along a parameter
// direction with d sigma, d mu (A = P (I - sigma_+^{-1}) since
// sigma_- = sigma_+ - I):
//   dA = P sigma_+^{-1} dsigma sigma_+^{-1}
//   db = P (sigma_+^{-1} dmu - sigma_+^{-1} dsigma sigma_+^{-1} mu)
//   dc = c [ -(dmu^dag S mu + mu^dag S dmu - mu^dag S dsigma S mu)/2
//            - tr(S dsigma)/2 ],  S = sigma_+^{-1}.
#include <cmath>
#include <complex>
#include <cstring>
#include <thread>
#include <vector>

#include "fk_internal.h"
#include "../../include/fockdiag.h"

namespace fk {
namespace {

using cd = std::complex<double>;
using Mat = std::vector<cd>;

Mat matmul(int n, const Mat &a, const Mat &b)
{
    Mat c((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k) {
            const cd aik = a[(size_t)i * n + k];
            if (aik == cd(0, 0)) continue;
            for (int j = 0; j < n; ++j) c[(size_t)i * n + j] += aik * b[(size_t)k * n + j];
        }
    return c;
}

Mat transpose(int n, const Mat &a)
{
    Mat t((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) t[(size_t)j * n + i] = a[(size_t)i * n + j];
    return t;
}

bool invert(int n, Mat a, Mat &inv, cd *det)
{
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    cd d = 1.0;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = std::abs(a[(size_t)col * n + col]);
        for (int r = col + 1; r < n; ++r)
            if (std::abs(a[(size_t)r * n + col]) > best) { best = std::abs(a[(size_t)r * n + col]); piv = r; }
        if (!(best > 0.0)) return false;
        if (piv != col) {
            for (int c = 0; c < n; ++c) {
                std::swap(a[(size_t)piv * n + c], a[(size_t)col * n + c]);
                std::swap(inv[(size_t)piv * n + c], inv[(size_t)col * n + c]);
            }
            d = -d;
        }
        const cd p = a[(size_t)col * n + col];
        d *= p;
        for (int c = 0; c < n; ++c) {
            a[(size_t)col * n + c] /= p;
            inv[(size_t)col * n + c] /= p;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const cd f = a[(size_t)r * n + col];
            if (f == cd(0, 0)) continue;
            for (int c = 0; c < n; ++c) {
                a[(size_t)r * n + c] -= f * a[(size_t)col * n + c];
                inv[(size_t)r * n + c] -= f * inv[(size_t)col * n + c];
            }
        }
    }
    *det = d;
    return true;
}

// Unitary of the interferometer and its derivative with respect to angle
// number `which` (0-based over the 2*nbs + M angles; -1 = no derivative).
Mat interferometer(int M, const double *ang, int which)
{
    Mat U((size_t)M * M, 0.0);
    for (int i = 0; i < M; ++i) U[(size_t)i * M + i] = 1.0;
    int bs = 0;
    for (int i = 0; i <= M - 2; ++i)
        for (int k = 0; k <= M - 2 - i; ++k, ++bs) {
            const double t = ang[2 * bs], ph = ang[2 * bs + 1];
            cd m00 = std::cos(t), m01 = -std::exp(cd(0, -ph)) * std::sin(t);
            cd m10 = std::exp(cd(0, ph)) * std::sin(t), m11 = std::cos(t);
            if (which == 2 * bs) {                  // d/dtheta
                m00 = -std::sin(t);
                m01 = -std::exp(cd(0, -ph)) * std::cos(t);
                m10 = std::exp(cd(0, ph)) * std::cos(t);
                m11 = -std::sin(t);
            } else if (which == 2 * bs + 1) {       // d/dphi
                m00 = 0.0;
                m01 = cd(0, 1) * std::exp(cd(0, -ph)) * std::sin(t);
                m10 = cd(0, 1) * std::exp(cd(0, ph)) * std::sin(t);
                m11 = 0.0;
            }
            // U <- T U, T acting on rows k, k+1
            for (int c = 0; c < M; ++c) {
                const cd a = U[(size_t)k * M + c], b = U[(size_t)(k + 1) * M + c];
                U[(size_t)k * M + c] = m00 * a + m01 * b;
                U[(size_t)(k + 1) * M + c] = m10 * a + m11 * b;
            }
            // a differentiated factor has zero rows outside (k, k+1)
            if (which == 2 * bs || which == 2 * bs + 1)
                for (int j = 0; j < M; ++j)
                    if (j != k && j != k + 1)
                        for (int c = 0; c < M; ++c) U[(size_t)j * M + c] = 0.0;
        }
    const double *psi = ang + 2 * bs;
    for (int j = 0; j < M; ++j) {
        cd f = std::exp(cd(0, psi[j]));
        if (which == 2 * bs + j) f *= cd(0, 1);
        for (int c = 0; c < M; ++c) U[(size_t)j * M + c] *= f;
    }
    if (which >= 2 * bs) {   // derivative of one phase: the other rows vanish
        for (int j = 0; j < M; ++j)
            if (which != 2 * bs + j)
                for (int c = 0; c < M; ++c) U[(size_t)j * M + c] = 0.0;
    }
    return U;
}

// Real symplectic [[Re U, -Im U], [Im U, Re U]] on (x.., p..).
std::vector<double> symplectic(int M, const Mat &U)
{
    const int n = 2 * M;
    std::vector<double> S((size_t)n * n, 0.0);
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            const cd u = U[(size_t)i * M + j];
            S[(size_t)i * n + j] = u.real();
            S[(size_t)i * n + M + j] = -u.imag();
            S[(size_t)(M + i) * n + j] = u.imag();
            S[(size_t)(M + i) * n + M + j] = u.real();
        }
    return S;
}

std::vector<double> rmul(int n, const std::vector<double> &a, const std::vector<double> &b)
{
    std::vector<double> c((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j) c[(size_t)i * n + j] += a[(size_t)i * n + k] * b[(size_t)k * n + j];
    return c;
}

std::vector<double> rtrans(int n, const std::vector<double> &a)
{
    std::vector<double> t((size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) t[(size_t)j * n + i] = a[(size_t)i * n + j];
    return t;
}

}  // namespace
}  // namespace fk

using namespace fk;

extern "C" int fk_circuit_triple(int M, const double *theta, double eta, fk_c128 *A, fk_c128 *b,
                                 fk_c128 *c, fk_c128 *dA, fk_c128 *db, fk_c128 *dc)
{
    if (M < 1 || M > 16 || !theta || !A || !b || !c || !(eta > 0.0) || eta > 1.0) return FK_EINVAL;
    const int n = 2 * M, P = M * M + 2 * M;
    const double *r = theta, *xd = theta + M, *ang = theta + 2 * M;
    try {
        // vacuum -> squeeze -> displace: V0, m0
        std::vector<double> V0((size_t)n * n, 0.0), m0(n, 0.0);
        for (int j = 0; j < M; ++j) {
            V0[(size_t)j * n + j] = 0.5 * std::exp(-2.0 * r[j]);
            V0[(size_t)(M + j) * n + M + j] = 0.5 * std::exp(2.0 * r[j]);
            m0[j] = std::sqrt(2.0) * xd[j];
        }
        const Mat U = interferometer(M, ang, -1);
        const std::vector<double> S = symplectic(M, U), St = rtrans(n, S);
        const double se = std::sqrt(eta);
        auto lossy = [&](const std::vector<double> &V) {   // X V X + (1-eta)/2 I
            std::vector<double> out(V.size());
            for (size_t i = 0; i < V.size(); ++i) out[i] = eta * V[i];
            return out;
        };
        std::vector<double> V = lossy(rmul(n, rmul(n, S, V0), St));
        for (int i = 0; i < n; ++i) V[(size_t)i * n + i] += 0.5 * (1.0 - eta);
        std::vector<double> mean(n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < n; ++k) mean[i] += se * S[(size_t)i * n + k] * m0[k];

        // complex covariance and mean: sigma = W V W^dag, mu = W mean
        const double r2 = 1.0 / std::sqrt(2.0);
        Mat W((size_t)n * n, 0.0);
        for (int j = 0; j < M; ++j) {
            W[(size_t)j * n + j] = r2;
            W[(size_t)j * n + M + j] = cd(0, r2);
            W[(size_t)(M + j) * n + j] = r2;
            W[(size_t)(M + j) * n + M + j] = cd(0, -r2);
        }
        auto to_sigma = [&](const std::vector<double> &Vr) {
            Mat s((size_t)n * n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int k = 0; k < n; ++k) {
                    cd acc = 0;
                    for (int l = 0; l < n; ++l)
                        for (int m = 0; m < n; ++m)
                            acc += W[(size_t)i * n + l] * Vr[(size_t)l * n + m] * std::conj(W[(size_t)k * n + m]);
                    s[(size_t)i * n + k] = acc;
                }
            return s;
        };
        auto to_mu = [&](const std::vector<double> &mr) {
            std::vector<cd> m(n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int l = 0; l < n; ++l) m[i] += W[(size_t)i * n + l] * mr[l];
            return m;
        };
        Mat sig = to_sigma(V);
        std::vector<cd> mu = to_mu(mean);
        Mat sp = sig;
        for (int i = 0; i < n; ++i) sp[(size_t)i * n + i] += 0.5;
        Mat Si;
        cd det;
        if (!invert(n, sp, Si, &det)) return FK_EINVAL;
        std::vector<cd> Smu(n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int l = 0; l < n; ++l) Smu[i] += Si[(size_t)i * n + l] * mu[l];
        cd q = 0;
        for (int i = 0; i < n; ++i) q += std::conj(mu[i]) * Smu[i];
        const cd cval = std::exp(-0.5 * q) / std::sqrt(det);
        // block-order A = P (I - S), b = P S mu; lattice order as fk_gaussian_to_triple
        std::vector<int> perm(n);
        for (int j = 0; j < M; ++j) {
            perm[2 * j] = M + j;
            perm[2 * j + 1] = j;
        }
        auto prow = [&](int i) { return (i + M) % n; };   // (P X)_{i,.} = X_{(i+M) mod n, .}
        for (int i = 0; i < n; ++i) {
            for (int k = 0; k < n; ++k) {
                const int bi = perm[i], bk = perm[k];
                const cd v = (prow(bi) == bk ? 1.0 : 0.0) - Si[(size_t)prow(bi) * n + bk];
                A[(size_t)i * n + k] = {v.real(), v.imag()};
            }
            const cd v = Smu[prow(perm[i])];
            b[i] = {v.real(), v.imag()};
        }
        *c = {cval.real(), cval.imag()};
        if (!dA && !db && !dc) return FK_OK;

        for (int p = 0; p < P; ++p) {
            // dV, dmean along parameter p
            std::vector<double> dV((size_t)n * n, 0.0), dmean(n, 0.0);
            if (p < M) {
                std::vector<double> dV0((size_t)n * n, 0.0);
                dV0[(size_t)p * n + p] = -std::exp(-2.0 * r[p]);
                dV0[(size_t)(M + p) * n + M + p] = std::exp(2.0 * r[p]);
                dV = lossy(rmul(n, rmul(n, S, dV0), St));
            } else if (p < 2 * M) {
                for (int i = 0; i < n; ++i) dmean[i] = se * S[(size_t)i * n + (p - M)] * std::sqrt(2.0);
            } else {
                const Mat dU = interferometer(M, ang, p - 2 * M);
                const std::vector<double> dS = symplectic(M, dU);
                const std::vector<double> a1 = rmul(n, rmul(n, dS, V0), St);
                std::vector<double> sum(a1.size());
                const std::vector<double> a1t = rtrans(n, a1);
                for (size_t i = 0; i < a1.size(); ++i) sum[i] = a1[i] + a1t[i];
                dV = lossy(sum);
                for (int i = 0; i < n; ++i)
                    for (int k = 0; k < n; ++k) dmean[i] += se * dS[(size_t)i * n + k] * m0[k];
            }
            const Mat dsig = to_sigma(dV);
            const std::vector<cd> dmu = to_mu(dmean);
            const Mat SdS = matmul(n, Si, dsig);
            const Mat SdSS = matmul(n, SdS, Si);
            std::vector<cd> dbb(n, 0.0);
            for (int i = 0; i < n; ++i) {
                cd acc = 0;
                for (int l = 0; l < n; ++l) acc += Si[(size_t)i * n + l] * dmu[l] - SdSS[(size_t)i * n + l] * mu[l];
                dbb[i] = acc;
            }
            cd t1 = 0, t2 = 0, t3 = 0, tr = 0;
            std::vector<cd> Sdmu(n, 0.0);
            for (int i = 0; i < n; ++i)
                for (int l = 0; l < n; ++l) Sdmu[i] += Si[(size_t)i * n + l] * dmu[l];
            for (int i = 0; i < n; ++i) {
                t1 += std::conj(dmu[i]) * Smu[i];
                t2 += std::conj(mu[i]) * Sdmu[i];
                cd s3 = 0;
                for (int l = 0; l < n; ++l) s3 += SdSS[(size_t)i * n + l] * mu[l];
                t3 += std::conj(mu[i]) * s3;
                tr += SdS[(size_t)i * n + i];
            }
            const cd dcv = cval * (-0.5 * (t1 + t2 - t3) - 0.5 * tr);
            for (int i = 0; i < n; ++i) {
                if (dA)
                    for (int k = 0; k < n; ++k) {
                        const cd v = SdSS[(size_t)prow(perm[i]) * n + perm[k]];
                        dA[((size_t)p * n + i) * n + k] = {v.real(), v.imag()};
                    }
                if (db) {
                    const cd v = dbb[prow(perm[i])];
                    db[(size_t)p * n + i] = {v.real(), v.imag()};
                }
            }
            if (dc) dc[p] = {dcv.real(), dcv.imag()};
        }
        return FK_OK;
    } catch (...) {
        return FK_ENOMEM;
    }
}

extern "C" int fk_circuit_triple_batched(int n, int M, const double *theta, double eta, fk_c128 *A,
                                         fk_c128 *b, fk_c128 *c, fk_c128 *dA, fk_c128 *db,
                                         fk_c128 *dc, int threads)
{
    if (n < 1 || M < 1 || M > 16 || !theta || !A || !b || !c) return FK_EINVAL;
    const int D = 2 * M, P = M * M + 2 * M;
    if (threads < 1) threads = (int)std::thread::hardware_concurrency();
    if (threads < 1) threads = 1;
    if (threads > n) threads = n;
    std::vector<int> status(threads, FK_OK);
    auto work = [&](int t) {
        for (int i = t; i < n; i += threads) {
            const int rc = fk_circuit_triple(M, theta + (size_t)i * P, eta, A + (size_t)i * D * D,
                                             b + (size_t)i * D, c + i,
                                             dA ? dA + (size_t)i * P * D * D : nullptr,
                                             db ? db + (size_t)i * P * D : nullptr,
                                             dc ? dc + (size_t)i * P : nullptr);
            if (rc) { status[t] = rc; return; }
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(work, t);
    work(0);
    for (auto &th : pool) th.join();
    for (int rc : status)
        if (rc) return rc;
    return FK_OK;
}
