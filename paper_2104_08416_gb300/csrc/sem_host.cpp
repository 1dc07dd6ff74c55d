// Host-side preprocessing (see sem_host.h). Built with -ffp-contract=off so
// that the floating-point steps that decide integers (Hilbert cells) round
// exactly as written.
#include "sem_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>
#include <unordered_map>
#include <atomic>
#include <thread>

namespace semhost {

namespace {
// f(begin, end) over contiguous chunks of [0, n) on up to 16 host threads
// (one thread when n is below `grain`); chunk t is [n t / T, n (t+1) / T).
template <class F>
void parallel_for(int64_t n, int64_t grain, F&& f) {
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int64_t T = std::max<int64_t>(1, std::min<int64_t>(hw, n / std::max<int64_t>(1, grain)));
    if (T <= 1) {
        f((int64_t)0, n, 0);
        return;
    }
    std::vector<std::thread> pool;
    for (int64_t t = 1; t < T; ++t) pool.emplace_back([&, t]() { f(n * t / T, n * (t + 1) / T, (int)t); });
    f((int64_t)0, n / T, 0);
    for (auto& th : pool) th.join();
}
int parallel_chunks(int64_t n, int64_t grain) {
    const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    return (int)std::max<int64_t>(1, std::min<int64_t>(hw, n / std::max<int64_t>(1, grain)));
}

// Local edges (slot s = 4 e + le, from corner le to le+1) grouped by their
// vertex pair without hashing: slots bucketed by the lower vertex in slot
// order, then matched on the higher vertex inside each (small) bucket.
// first[s] = the lowest slot holding the same edge; returns the largest
// number of slots sharing one edge.
int group_edges(const int32_t* quads, int64_t ne, int64_t nv, std::vector<int64_t>& first) {
    const int64_t ns = ne * 4;
    std::vector<int64_t> ptr((size_t)nv + 1, 0);
    for (int64_t s = 0; s < ns; ++s) {
        const int32_t a = quads[s], b = quads[(s & ~int64_t(3)) + ((s + 1) & 3)];
        ptr[(size_t)std::min(a, b) + 1]++;
    }
    for (size_t k = 1; k < ptr.size(); ++k) ptr[k] += ptr[k - 1];
    std::vector<int64_t> bucket((size_t)ns);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t s = 0; s < ns; ++s) {
            const int32_t a = quads[s], b = quads[(s & ~int64_t(3)) + ((s + 1) & 3)];
            bucket[(size_t)fill[(size_t)std::min(a, b)]++] = s;
        }
    }
    first.assign((size_t)ns, -1);
    std::vector<int> mult(parallel_chunks(nv, 1 << 15), 0);
    parallel_for(nv, 1 << 15, [&](int64_t v0, int64_t v1, int t) {
        int mx = 0;
        for (int64_t v = v0; v < v1; ++v)
            for (int64_t i = ptr[(size_t)v]; i < ptr[(size_t)v + 1]; ++i) {
                const int64_t s = bucket[(size_t)i];
                const int32_t hs = std::max(quads[s], quads[(s & ~int64_t(3)) + ((s + 1) & 3)]);
                int64_t f = s;
                int cnt = 0;
                for (int64_t j = ptr[(size_t)v]; j < ptr[(size_t)v + 1]; ++j) {
                    const int64_t r = bucket[(size_t)j];
                    if (std::max(quads[r], quads[(r & ~int64_t(3)) + ((r + 1) & 3)]) == hs) {
                        if (cnt == 0) f = r;  // the bucket is in slot order
                        ++cnt;
                    }
                }
                first[(size_t)s] = f;
                mx = std::max(mx, cnt);
            }
        mult[(size_t)t] = mx;
    });
    return *std::max_element(mult.begin(), mult.end());
}
}  // namespace

// ---------------------------------------------------------------- GLL rule
static void legendre_eval(int p, double x, double& Pp, double& Pm1) {
    double a = 1.0, b = x;  // P_0, P_1
    if (p == 0) { Pp = 1.0; Pm1 = 0.0; return; }
    for (int k = 1; k < p; ++k) {
        double c = ((2.0 * k + 1.0) * x * b - k * a) / (k + 1.0);
        a = b;
        b = c;
    }
    Pp = b;
    Pm1 = a;
}

void gll_rule(int p, std::vector<double>& x, std::vector<double>& w) {
    const int n = p + 1;
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    x[0] = -1.0;
    x[p] = 1.0;
    // interior nodes: roots of P_p', Newton from the Chebyshev-Lobatto points
    for (int k = 1; k < p; ++k) {
        double t = -std::cos(M_PI * k / p);
        for (int it = 0; it < 100; ++it) {
            double Pp, Pm1;
            legendre_eval(p, t, Pp, Pm1);
            double d1 = p * (t * Pp - Pm1) / (t * t - 1.0);                 // P_p'
            double d2 = (2.0 * t * d1 - p * (p + 1.0) * Pp) / (1.0 - t * t);  // P_p''
            double dt = d1 / d2;
            t -= dt;
            if (std::fabs(dt) < 1e-17) break;
        }
        x[k] = t;
    }
    std::vector<double> s(x);
    for (int k = 0; k < n; ++k) x[k] = 0.5 * (s[k] - s[p - k]);
    for (int k = 0; k < n; ++k) {
        double Pp, Pm1;
        legendre_eval(p, x[k], Pp, Pm1);
        w[k] = 2.0 / (p * (p + 1.0) * Pp * Pp);
    }
}

void gll_derivative(const std::vector<double>& x, std::vector<double>& D) {
    // Closed form for the GLL collocation derivative (e.g. Canuto, Hussaini,
    // Quarteroni & Zang, Spectral Methods, eq. 2.4.34):
    // D_ij = P_p(x_i) / (P_p(x_j) (x_i - x_j)) for i != j, D_00 = -p(p+1)/4,
    // D_pp = p(p+1)/4, other diagonal entries 0.
    const int n = (int)x.size();
    const int p = n - 1;
    std::vector<double> L(n);
    for (int i = 0; i < n; ++i) {
        double Pp, Pm1;
        legendre_eval(p, x[i], Pp, Pm1);
        L[i] = Pp;
    }
    D.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (i != j) D[(size_t)i * n + j] = L[i] / (L[j] * (x[i] - x[j]));
    if (p >= 1) {
        D[0] = -p * (p + 1.0) / 4.0;
        D[(size_t)p * n + p] = p * (p + 1.0) / 4.0;
    }
}

// --------------------------------------------------------------- geometry
// Bilinear map X(xi, eta) = a + b xi + c eta + d xi eta of a quad with
// counter-clockwise corners X0..X3 at (-1,-1), (1,-1), (1,1), (-1,1).
static inline void jac_at(const double* X, double xi, double eta, double J[4]) {
    // columns: dX/dxi, dX/deta
    for (int a = 0; a < 2; ++a) {
        double x0 = X[0 * 2 + a], x1 = X[1 * 2 + a], x2 = X[2 * 2 + a], x3 = X[3 * 2 + a];
        J[a * 2 + 0] = 0.25 * ((x1 - x0) * (1.0 - eta) + (x2 - x3) * (1.0 + eta));
        J[a * 2 + 1] = 0.25 * ((x3 - x0) * (1.0 - xi) + (x2 - x1) * (1.0 + xi));
    }
}

std::string validate(const double* coords, int64_t nv, const int32_t* quads, int64_t ne, int p) {
    if (nv <= 0 || ne <= 0) return "empty mesh";
    if (p < 1 || p > 8) return "order must be in 1..8";
    std::vector<uint8_t> used((size_t)nv, 0);
    for (int64_t i = 0; i < ne * 4; ++i) {
        int32_t v = quads[i];
        if (v < 0 || v >= nv) return "quad vertex index out of range";
        used[(size_t)v] = 1;
    }
    for (int64_t v = 0; v < nv; ++v)
        if (!used[(size_t)v]) return "unreferenced vertex " + std::to_string(v);
    for (int64_t i = 0; i < nv * 2; ++i)
        if (!std::isfinite(coords[i])) return "non-finite coordinate";
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* q = quads + e * 4;
        for (int a = 0; a < 4; ++a)
            for (int b = a + 1; b < 4; ++b)
                if (q[a] == q[b]) return "quad " + std::to_string(e) + " repeats a vertex";
    }
    {
        std::vector<int64_t> first;
        if (group_edges(quads, ne, nv, first) > 2) return "edge shared by more than two quads";
    }
    std::vector<double> x, w;
    gll_rule(p, x, w);
    // the first element (lowest id) with a non-positive Jacobian
    std::vector<int64_t> bad(parallel_chunks(ne, 1 << 14), ne);
    parallel_for(ne, 1 << 14, [&](int64_t e0, int64_t e1, int t) {
        for (int64_t e = e0; e < e1; ++e) {
            double X[8];
            for (int c = 0; c < 4; ++c) {
                X[c * 2 + 0] = coords[(size_t)quads[e * 4 + c] * 2 + 0];
                X[c * 2 + 1] = coords[(size_t)quads[e * 4 + c] * 2 + 1];
            }
            for (int j = 0; j <= p; ++j)
                for (int i = 0; i <= p; ++i) {
                    double J[4];
                    jac_at(X, x[i], x[j], J);
                    const double det = J[0] * J[3] - J[1] * J[2];
                    if (!(det > 0.0)) {
                        bad[(size_t)t] = e;
                        return;
                    }
                }
        }
    });
    const int64_t e_bad = *std::min_element(bad.begin(), bad.end());
    if (e_bad < ne) return "non-positive Jacobian in quad " + std::to_string(e_bad) + " (clockwise or degenerate)";
    return "";
}

// ------------------------------------------------------- canonical numbering
void number_nodes(Mesh& m) {
    const int p = m.p, n = p + 1, P = n * n;
    m.np = n;
    m.P = P;
    m.conn.assign((size_t)m.ne * P, -1);
    m.edge_lo.clear();
    m.edge_hi.clear();
    m.edge_first.clear();
    const int corner[4] = {0, p, p * n + p, p * n};
    int64_t next = m.nv;
    // pass 1: edges in order of first appearance (slot order)
    std::vector<int64_t> eid((size_t)m.ne * 4);
    {
        std::vector<int64_t> first;
        group_edges(m.quads.data(), m.ne, m.nv, first);
        for (int64_t s = 0; s < m.ne * 4; ++s) {
            if (first[(size_t)s] == s) {
                const int64_t va = m.quads[(size_t)s], vb = m.quads[(size_t)((s & ~int64_t(3)) + ((s + 1) & 3))];
                eid[(size_t)s] = (int64_t)m.edge_lo.size();
                m.edge_lo.push_back(std::min(va, vb));
                m.edge_hi.push_back(std::max(va, vb));
                m.edge_first.push_back(next);
                next += p - 1;
            } else {
                eid[(size_t)s] = eid[(size_t)first[(size_t)s]];
            }
        }
    }
    const int64_t interior0 = next;
    parallel_for(m.ne, 1 << 14, [&](int64_t e0, int64_t e1, int) {
    for (int64_t e = e0; e < e1; ++e) {
        const int32_t* q = &m.quads[(size_t)e * 4];
        int32_t* c = &m.conn[(size_t)e * P];
        for (int k = 0; k < 4; ++k) c[corner[k]] = q[k];
        for (int le = 0; le < 4; ++le) {
            int64_t id = eid[(size_t)e * 4 + le];
            bool forward = q[le] < q[(le + 1) & 3];  // walking from lower to higher id
            for (int t = 1; t < p; ++t) {
                // t-th interior point from the edge's first corner
                int li;
                if (le == 0) li = t;
                else if (le == 1) li = t * n + p;
                else if (le == 2) li = p * n + (p - t);
                else li = (p - t) * n;
                int k = forward ? t : p - t;  // position counted from the lower vertex
                c[li] = (int32_t)(m.edge_first[(size_t)id] + (k - 1));
            }
        }
        // element-interior nodes: elements ascending, i fastest
        const int64_t base = interior0 + e * (int64_t)(p - 1) * (p - 1);
        for (int j = 1; j < p; ++j)
            for (int i = 1; i < p; ++i) c[j * n + i] = (int32_t)(base + (j - 1) * (p - 1) + (i - 1));
    }
    });
    m.nn = interior0 + m.ne * (int64_t)(p - 1) * (p - 1);
}

void node_coordinates(const Mesh& m, std::vector<double>& xy) {
    std::vector<double> x, w;
    gll_rule(m.p, x, w);
    const int p = m.p, n = p + 1;
    xy.assign((size_t)m.nn * 2, 0.0);
    for (size_t i = 0; i < (size_t)m.nv * 2; ++i) xy[i] = m.coords[i];
    parallel_for((int64_t)m.edge_lo.size(), 1 << 15, [&](int64_t d0, int64_t d1, int) {
    for (int64_t ed = d0; ed < d1; ++ed) {
        const double* A = &m.coords[(size_t)m.edge_lo[(size_t)ed] * 2];
        const double* B = &m.coords[(size_t)m.edge_hi[(size_t)ed] * 2];
        for (int k = 1; k < p; ++k) {
            double s = x[k];
            int64_t id = m.edge_first[(size_t)ed] + k - 1;
            xy[(size_t)id * 2 + 0] = 0.5 * ((1.0 - s) * A[0] + (1.0 + s) * B[0]);
            xy[(size_t)id * 2 + 1] = 0.5 * ((1.0 - s) * A[1] + (1.0 + s) * B[1]);
        }
    }
    });
    parallel_for(m.ne, 1 << 14, [&](int64_t e0, int64_t e1, int) {
    for (int64_t e = e0; e < e1; ++e) {
        const int32_t* q = &m.quads[(size_t)e * 4];
        const int32_t* c = &m.conn[(size_t)e * m.P];
        for (int j = 1; j < p; ++j)
            for (int i = 1; i < p; ++i) {
                double xi = x[i], eta = x[j];
                double f0 = 0.25 * (1 - xi) * (1 - eta), f1 = 0.25 * (1 + xi) * (1 - eta);
                double f2 = 0.25 * (1 + xi) * (1 + eta), f3 = 0.25 * (1 - xi) * (1 + eta);
                for (int a = 0; a < 2; ++a) {
                    double v = ((f0 * m.coords[(size_t)q[0] * 2 + a] + f1 * m.coords[(size_t)q[1] * 2 + a]) +
                                f2 * m.coords[(size_t)q[2] * 2 + a]) +
                               f3 * m.coords[(size_t)q[3] * 2 + a];
                    xy[(size_t)c[j * n + i] * 2 + a] = v;
                }
            }
    }
    });
}

// ------------------------------------------------ generalized Hilbert curve
// The construction of Cerveny's generalized Hilbert ("gilbert") curve, which
// Section 3 cites for rectangles of any side lengths, with this library's own
// parity rules and top-level orientation. Recursive split of a w x h block spanned by the integer vectors A (length w
// along the curve's main direction) and B (length h), starting at origin O
// and ending at O + (w-1) a. Long blocks (2w > 3h) are cut in two along A
// (first part even when h is even); otherwise the block is cut into a
// transposed lower-left part, the full-width upper part and a reversed
// lower-right part, with the cut height made even so that every part admits a
// path between the required corners.
namespace {
struct Frame {
    int64_t ox, oy, ax, ay, bx, by;
};
inline int64_t sgn(int64_t v) { return (v > 0) - (v < 0); }
}  // namespace

void hilbert_cells(int64_t W, int64_t H, std::vector<int32_t>& cells) {
    cells.clear();
    cells.reserve((size_t)(W * H * 2));
    std::vector<Frame> st;
    if ((W & 1) && !(H & 1)) st.push_back({0, 0, 0, H, W, 0});
    else st.push_back({0, 0, W, 0, 0, H});
    while (!st.empty()) {
        Frame f = st.back();
        st.pop_back();
        int64_t w = std::llabs(f.ax) + std::llabs(f.ay), h = std::llabs(f.bx) + std::llabs(f.by);
        int64_t dax = sgn(f.ax), day = sgn(f.ay), dbx = sgn(f.bx), dby = sgn(f.by);
        if (h == 1) {
            for (int64_t i = 0; i < w; ++i) {
                cells.push_back((int32_t)(f.ox + i * dax));
                cells.push_back((int32_t)(f.oy + i * day));
            }
            continue;
        }
        if (w == 1) {
            for (int64_t j = 0; j < h; ++j) {
                cells.push_back((int32_t)(f.ox + j * dbx));
                cells.push_back((int32_t)(f.oy + j * dby));
            }
            continue;
        }
        if (2 * w > 3 * h) {
            int64_t w1 = w / 2;
            if ((h % 2 == 0) && (w1 % 2 == 1) && w1 > 1) w1 -= 1;
            Frame second{f.ox + w1 * dax, f.oy + w1 * day, (w - w1) * dax, (w - w1) * day, f.bx, f.by};
            Frame first{f.ox, f.oy, w1 * dax, w1 * day, f.bx, f.by};
            st.push_back(second);
            st.push_back(first);
        } else {
            int64_t h1 = h / 2;
            if ((h1 % 2 == 1) && h > 2) h1 += 1;
            int64_t w1 = w / 2;
            Frame lowleft{f.ox, f.oy, h1 * dbx, h1 * dby, w1 * dax, w1 * day};
            Frame upper{f.ox + h1 * dbx, f.oy + h1 * dby, f.ax, f.ay, (h - h1) * dbx, (h - h1) * dby};
            Frame lowright{f.ox + (w - 1) * dax + (h1 - 1) * dbx, f.oy + (w - 1) * day + (h1 - 1) * dby,
                           -h1 * dbx, -h1 * dby, -(w - w1) * dax, -(w - w1) * day};
            st.push_back(lowright);
            st.push_back(upper);
            st.push_back(lowleft);
        }
    }
}

// ------------------------------------------------------------- orderings
static int64_t ceil_sqrt(int64_t n) {
    int64_t r = (int64_t)std::sqrt((double)n);
    while (r * r > n) --r;
    while ((r + 1) * (r + 1) <= n) ++r;
    return r * r == n ? r : r + 1;
}

std::string element_order_hilbert(const Mesh& m, std::vector<int64_t>& order, bool wide) {
    // Section 4.3: element centroids on a W x H grid over the bounding box,
    // cells walked along the curve, elements of a cell appended in input order.
    // Box sizes: W = ceil(sqrt(E)), H = max(1, ceil(W / r)); or, with `wide`,
    // the alternative the section gives for changing how many elements fall
    // in a cell (w_b = sqrt(E) r, h_b = sqrt(E)): H = ceil(sqrt(E)),
    // W = max(1, ceil(H r)). r = w_m / h_m in FP64.
    double xmin = std::numeric_limits<double>::infinity(), ymin = xmin;
    double xmax = -xmin, ymax = -xmin;
    for (int64_t v = 0; v < m.nv; ++v) {
        xmin = std::min(xmin, m.coords[(size_t)v * 2]);
        xmax = std::max(xmax, m.coords[(size_t)v * 2]);
        ymin = std::min(ymin, m.coords[(size_t)v * 2 + 1]);
        ymax = std::max(ymax, m.coords[(size_t)v * 2 + 1]);
    }
    const double wm = xmax - xmin, hm = ymax - ymin;
    const double r = wm / hm;
    int64_t W, H;
    if (!wide) {
        W = ceil_sqrt(m.ne);
        H = std::max<int64_t>(1, (int64_t)std::ceil((double)W / r));
    } else {
        H = ceil_sqrt(m.ne);
        const double wd = std::ceil((double)H * r);
        if (!(wd < 2147483647.0)) return "Hilbert grid too large for this aspect ratio";
        W = std::max<int64_t>(1, (int64_t)wd);
    }
    if (W * H > 2147483647LL / 2) return "Hilbert grid too large for this aspect ratio";
    std::vector<int32_t> cells;
    hilbert_cells(W, H, cells);
    std::vector<int64_t> rank((size_t)(W * H));
    for (int64_t k = 0; k < W * H; ++k) rank[(size_t)(cells[k * 2] * H + cells[k * 2 + 1])] = k;
    std::vector<int64_t> key((size_t)m.ne);
    for (int64_t e = 0; e < m.ne; ++e) {
        const int32_t* q = &m.quads[(size_t)e * 4];
        double xs = (m.coords[(size_t)q[0] * 2] + m.coords[(size_t)q[1] * 2]) +
                    (m.coords[(size_t)q[2] * 2] + m.coords[(size_t)q[3] * 2]);
        double ys = (m.coords[(size_t)q[0] * 2 + 1] + m.coords[(size_t)q[1] * 2 + 1]) +
                    (m.coords[(size_t)q[2] * 2 + 1] + m.coords[(size_t)q[3] * 2 + 1]);
        double xc = xs * 0.25, yc = ys * 0.25;
        double fx = std::floor(((xc - xmin) * (double)W) / wm);
        double fy = std::floor(((yc - ymin) * (double)H) / hm);
        int64_t ix = std::max<int64_t>(0, std::min<int64_t>(W - 1, (int64_t)fx));
        int64_t iy = std::max<int64_t>(0, std::min<int64_t>(H - 1, (int64_t)fy));
        key[(size_t)e] = rank[(size_t)(ix * H + iy)];
    }
    // stable counting sort by curve position
    std::vector<int64_t> cnt((size_t)(W * H + 1), 0);
    for (int64_t e = 0; e < m.ne; ++e) cnt[(size_t)key[(size_t)e] + 1]++;
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    order.assign((size_t)m.ne, 0);
    for (int64_t e = 0; e < m.ne; ++e) order[(size_t)cnt[(size_t)key[(size_t)e]]++] = e;
    return "";
}

void node_degrees(const Mesh& m, std::vector<int32_t>& deg) {
    // degree = number of distinct other nodes sharing an element. Nodes of one
    // element only have P-1; all interior nodes of an edge share one element
    // set, so one evaluation per edge and per vertex suffices.
    const int P = m.P, p = m.p;
    deg.assign((size_t)m.nn, P - 1);
    // vertex -> elements
    std::vector<int64_t> vptr((size_t)m.nv + 1, 0);
    for (int64_t i = 0; i < m.ne * 4; ++i) vptr[(size_t)m.quads[(size_t)i] + 1]++;
    for (size_t k = 1; k < vptr.size(); ++k) vptr[k] += vptr[k - 1];
    std::vector<int64_t> vel((size_t)(m.ne * 4));
    {
        std::vector<int64_t> fill(vptr.begin(), vptr.end() - 1);
        for (int64_t e = 0; e < m.ne; ++e)
            for (int c = 0; c < 4; ++c) vel[(size_t)fill[(size_t)m.quads[(size_t)e * 4 + c]]++] = e;
    }
    // distinct nodes of a few elements, minus one
    auto count_union = [&](const int64_t* els, int k, std::vector<int32_t>& buf) {
        buf.clear();
        for (int t = 0; t < k; ++t) {
            const int32_t* cc = &m.conn[(size_t)els[t] * P];
            buf.insert(buf.end(), cc, cc + P);
        }
        std::sort(buf.begin(), buf.end());
        return (int32_t)(std::unique(buf.begin(), buf.end()) - buf.begin()) - 1;
    };
    parallel_for(m.nv, 1 << 14, [&](int64_t v0, int64_t v1, int) {
        std::vector<int32_t> buf;
        for (int64_t v = v0; v < v1; ++v)
            deg[(size_t)v] =
                count_union(&vel[(size_t)vptr[(size_t)v]], (int)(vptr[(size_t)v + 1] - vptr[(size_t)v]), buf);
    });
    if (p >= 2) {
        // elements of an edge = elements holding both of its vertices
        parallel_for((int64_t)m.edge_lo.size(), 1 << 14, [&](int64_t d0, int64_t d1, int) {
            std::vector<int32_t> buf;
            for (int64_t ed = d0; ed < d1; ++ed) {
                const int64_t a = m.edge_lo[(size_t)ed], b = m.edge_hi[(size_t)ed];
                int64_t els[8];
                int k = 0;
                for (int64_t t = vptr[(size_t)a]; t < vptr[(size_t)a + 1]; ++t) {
                    const int64_t e = vel[(size_t)t];
                    const int32_t* q = &m.quads[(size_t)e * 4];
                    for (int c = 0; c < 4; ++c) {
                        if (q[c] == b && (q[(c + 1) & 3] == a || q[(c + 3) & 3] == a)) {
                            if (k < 8) els[k++] = e;
                            break;
                        }
                    }
                }
                const int32_t d = count_union(els, k, buf);
                for (int t = 1; t < p; ++t) deg[(size_t)(m.edge_first[(size_t)ed] + t - 1)] = d;
            }
        });
    }
}

void renumber_nodes(const Mesh& m, const std::vector<int64_t>& elem_order, const std::vector<int32_t>& deg,
                    std::vector<int64_t>& node_order) {
    // Section 4.3 node procedure: first touch along the element order, each
    // element's new nodes sorted by ascending degree (stable).
    const int P = m.P;
    std::vector<uint8_t> seen((size_t)m.nn, 0);
    node_order.clear();
    node_order.reserve((size_t)m.nn);
    std::vector<int64_t> group;
    group.reserve((size_t)P);
    for (int64_t e : elem_order) {
        group.clear();
        const int32_t* c = &m.conn[(size_t)e * P];
        for (int q = 0; q < P; ++q)
            if (!seen[(size_t)c[q]]) {
                seen[(size_t)c[q]] = 1;
                group.push_back(c[q]);
            }
        // stable insertion sort by degree (at most P nodes; no allocation)
        for (size_t i = 1; i < group.size(); ++i) {
            const int64_t x = group[i];
            const int32_t dx = deg[(size_t)x];
            size_t j = i;
            for (; j > 0 && deg[(size_t)group[j - 1]] > dx; --j) group[j] = group[j - 1];
            group[j] = x;
        }
        node_order.insert(node_order.end(), group.begin(), group.end());
    }
}

static inline uint64_t splitmix_next(uint64_t& s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

void random_order(int64_t n, uint64_t seed, std::vector<int64_t>& order) {
    order.resize((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    uint64_t s = seed;
    for (int64_t i = n - 1; i >= 1; --i) {
        uint64_t j = splitmix_next(s) % (uint64_t)(i + 1);
        std::swap(order[(size_t)i], order[(size_t)j]);
    }
}

// Node walks of Section 6.1's "Node Connectivity" (kind 4) and "Node
// Distance" (kind 5) strategies. Nodes are connected when they share an
// element. The walk starts at the best node (fewest connections, or closest to
// the lower-left corner of the bounding box; ties to the lower id) and
// repeatedly moves to the best unvisited node connected to the
// current one; at a dead end it backs up along the walk to the latest node
// that still has an unvisited connected node, and when the walk has visited
// its whole connected part it restarts at the best unvisited node. Visiting a
// node appends it to the node order and appends the elements that contain it
// (ascending id, each once) to the element order.
void walk_orders(const Mesh& m, int kind, std::vector<int64_t>& eo, std::vector<int64_t>& no) {
    const int P = m.P;
    const int64_t nn = m.nn, ne = m.ne;
    std::vector<int64_t> nptr((size_t)nn + 1, 0);
    for (int64_t s = 0; s < ne * P; ++s) nptr[(size_t)m.conn[(size_t)s] + 1]++;
    for (size_t k = 1; k < nptr.size(); ++k) nptr[k] += nptr[k - 1];
    std::vector<int64_t> nel((size_t)(ne * P));
    {
        std::vector<int64_t> fill(nptr.begin(), nptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int q = 0; q < P; ++q) nel[(size_t)fill[(size_t)m.conn[(size_t)(e * P + q)]]++] = e;
    }
    // integer keys: the number of connections, or the squared distance to the
    // reference point in units of 2^-30 of the bounding-box diagonal squared
    // (floor), so that nodes at mirror-equal distances tie exactly whatever the
    // last bit of their coordinates
    std::vector<int64_t> key((size_t)nn);
    if (kind == 4) {
        std::vector<int32_t> deg;
        node_degrees(m, deg);
        for (int64_t g = 0; g < nn; ++g) key[(size_t)g] = deg[(size_t)g];
    } else {
        std::vector<double> xy;
        node_coordinates(m, xy);
        double x0 = std::numeric_limits<double>::infinity(), y0 = x0, x1 = -x0, y1 = -x0;
        for (int64_t v = 0; v < m.nv; ++v) {
            x0 = std::min(x0, m.coords[(size_t)v * 2]);
            y0 = std::min(y0, m.coords[(size_t)v * 2 + 1]);
            x1 = std::max(x1, m.coords[(size_t)v * 2]);
            y1 = std::max(y1, m.coords[(size_t)v * 2 + 1]);
        }
        const double diag2 = (x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0);
        for (int64_t g = 0; g < nn; ++g) {
            const double dx = xy[(size_t)g * 2] - x0, dy = xy[(size_t)g * 2 + 1] - y0;
            key[(size_t)g] = (int64_t)std::floor((dx * dx + dy * dy) / diag2 * 1073741824.0);
        }
    }
    auto better = [&](int64_t a, int64_t b) {
        return key[(size_t)a] < key[(size_t)b] || (key[(size_t)a] == key[(size_t)b] && a < b);
    };
    std::vector<int64_t> by_key((size_t)nn);
    std::iota(by_key.begin(), by_key.end(), 0);
    std::sort(by_key.begin(), by_key.end(), [&](int64_t a, int64_t b) { return better(a, b); });
    std::vector<uint8_t> visited((size_t)nn, 0), listed((size_t)ne, 0);
    eo.clear();
    no.clear();
    eo.reserve((size_t)ne);
    no.reserve((size_t)nn);
    auto visit = [&](int64_t g) {
        visited[(size_t)g] = 1;
        no.push_back(g);
        for (int64_t k = nptr[(size_t)g]; k < nptr[(size_t)g + 1]; ++k) {
            const int64_t e = nel[(size_t)k];
            if (!listed[(size_t)e]) {
                listed[(size_t)e] = 1;
                eo.push_back(e);
            }
        }
    };
    std::vector<int64_t> stack;
    size_t cursor = 0;
    while ((int64_t)no.size() < nn) {
        while (visited[(size_t)by_key[cursor]]) ++cursor;
        visit(by_key[cursor]);
        stack.assign(1, by_key[cursor]);
        while (!stack.empty()) {
            const int64_t top = stack.back();
            int64_t best = -1;
            for (int64_t k = nptr[(size_t)top]; k < nptr[(size_t)top + 1]; ++k) {
                const int32_t* c = &m.conn[(size_t)nel[(size_t)k] * P];
                for (int q = 0; q < P; ++q) {
                    const int64_t g = c[q];
                    if (!visited[(size_t)g] && (best < 0 || better(g, best))) best = g;
                }
            }
            if (best < 0) {
                stack.pop_back();
            } else {
                visit(best);
                stack.push_back(best);
            }
        }
    }
}

std::string orderings(const Mesh& m, int kind, uint64_t seed, std::vector<int64_t>& eo, std::vector<int64_t>& no) {
    if (kind == 4 || kind == 5) {
        walk_orders(m, kind, eo, no);
        return "";
    }
    if (kind == 0) {
        eo.resize((size_t)m.ne);
        std::iota(eo.begin(), eo.end(), 0);
        no.resize((size_t)m.nn);
        std::iota(no.begin(), no.end(), 0);
        return "";
    }
    if (kind == 2) {
        random_order(m.ne, seed + 2, eo);
        random_order(m.nn, seed + 3, no);
        return "";
    }
    if (kind == 1) {
        eo.resize((size_t)m.ne);
        std::iota(eo.begin(), eo.end(), 0);
    } else {
        std::string why = element_order_hilbert(m, eo, kind == 6);
        if (!why.empty()) return why;
    }
    std::vector<int32_t> deg;
    node_degrees(m, deg);
    renumber_nodes(m, eo, deg, no);
    return "";
}

int64_t snap(const std::vector<double>& xy, double x, double y) {
    std::vector<int64_t> out;
    snap_many(xy, &x, &y, 1, 1, out);
    return out[0];
}

void snap_many(const std::vector<double>& xy, const double* qx, const double* qy, int64_t nq, int64_t stride,
               std::vector<int64_t>& out) {
    // every thread scans a contiguous node range for all points (a range
    // stays in cache across the points); the ranges' minima are combined in
    // range order with the same strict comparison, so a tie keeps the lowest id
    const int64_t n = (int64_t)(xy.size() / 2);
    const int T = parallel_chunks(n, 1 << 16);
    std::vector<double> bd((size_t)T * nq, std::numeric_limits<double>::infinity());
    std::vector<int64_t> bi((size_t)T * nq, 0);
    parallel_for(n, 1 << 16, [&](int64_t i0, int64_t i1, int t) {
        double* d = &bd[(size_t)t * nq];
        int64_t* b = &bi[(size_t)t * nq];
        for (int64_t c0 = i0; c0 < i1; c0 += 4096) {
            const int64_t c1 = std::min(i1, c0 + 4096);
            for (int64_t k = 0; k < nq; ++k) {
                const double x = qx[k * stride], y = qy[k * stride];
                for (int64_t i = c0; i < c1; ++i) {
                    const double dx = xy[(size_t)i * 2] - x, dy = xy[(size_t)i * 2 + 1] - y;
                    const double dd = dx * dx + dy * dy;
                    if (dd < d[k]) {
                        d[k] = dd;
                        b[k] = i;
                    }
                }
            }
        }
    });
    out.assign((size_t)nq, 0);
    for (int64_t k = 0; k < nq; ++k) {
        double best = std::numeric_limits<double>::infinity();
        for (int t = 0; t < T; ++t)
            if (bd[(size_t)t * nq + k] < best) {
                best = bd[(size_t)t * nq + k];
                out[(size_t)k] = bi[(size_t)t * nq + k];
            }
    }
}

double cfl_dt(const Mesh& m, const double* vel) {
    std::vector<double> x, w;
    gll_rule(m.p, x, w);
    const int n = m.p + 1;
    std::vector<double> part(parallel_chunks(m.ne, 1 << 14), std::numeric_limits<double>::infinity());
    parallel_for(m.ne, 1 << 14, [&](int64_t e0, int64_t e1, int th) {
    double best = std::numeric_limits<double>::infinity();
    std::vector<double> pts((size_t)n * n * 2);
    for (int64_t e = e0; e < e1; ++e) {
        const int32_t* q = &m.quads[(size_t)e * 4];
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                double xi = x[i], eta = x[j];
                double f0 = 0.25 * (1 - xi) * (1 - eta), f1 = 0.25 * (1 + xi) * (1 - eta);
                double f2 = 0.25 * (1 + xi) * (1 + eta), f3 = 0.25 * (1 - xi) * (1 + eta);
                for (int a = 0; a < 2; ++a)
                    pts[((size_t)j * n + i) * 2 + a] =
                        ((f0 * m.coords[(size_t)q[0] * 2 + a] + f1 * m.coords[(size_t)q[1] * 2 + a]) +
                         f2 * m.coords[(size_t)q[2] * 2 + a]) +
                        f3 * m.coords[(size_t)q[3] * 2 + a];
            }
        double dmin = std::numeric_limits<double>::infinity();
        for (int j = 0; j < n; ++j)
            for (int i = 0; i + 1 < n; ++i) {
                const double* A = &pts[((size_t)j * n + i) * 2];
                const double* B = &pts[((size_t)j * n + i + 1) * 2];
                dmin = std::min(dmin, std::hypot(B[0] - A[0], B[1] - A[1]));
            }
        for (int j = 0; j + 1 < n; ++j)
            for (int i = 0; i < n; ++i) {
                const double* A = &pts[((size_t)j * n + i) * 2];
                const double* B = &pts[((size_t)(j + 1) * n + i) * 2];
                dmin = std::min(dmin, std::hypot(B[0] - A[0], B[1] - A[1]));
            }
        best = std::min(best, dmin / vel[e]);
    }
    part[(size_t)th] = best;
    });
    return *std::min_element(part.begin(), part.end());
}

// ------------------------------------------------------------ block plan
static inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

std::string build_block_plan(const std::vector<int32_t>& conn, int64_t ne, int P, int64_t nn, int eb,
                             bool allow_dense, int vec, const std::vector<int32_t>& rec_gid, BlockPlan& pl) {
    using namespace semplan;
    pl = BlockPlan();
    pl.eb = eb;
    pl.P = P;
    pl.ne = ne;
    pl.nn = nn;
    if (eb < 1 || (int64_t)eb * P > 65535) return "elements per block outside 1 .. 65535 / points per element";
    pl.nblocks = (ne + eb - 1) / eb;
    const int64_t nb = pl.nblocks;
    // blocks touching each node (blocks are visited in ascending order)
    std::vector<int32_t> nblk((size_t)nn, 0);
    {
        std::vector<int32_t> last((size_t)nn, -1);
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t s1 = std::min(ne, (b + 1) * eb) * P;
            for (int64_t s = b * eb * P; s < s1; ++s) {
                const int32_t g = conn[(size_t)s];
                if (last[(size_t)g] != (int32_t)b) {
                    last[(size_t)g] = (int32_t)b;
                    nblk[(size_t)g]++;
                }
            }
        }
    }
    // DENSE when the nodes first touched by each block are the next id range
    bool dense = allow_dense;
    if (dense) {
        std::vector<uint8_t> seen((size_t)nn, 0);
        int64_t next = 0;
        for (int64_t b = 0; b < nb && dense; ++b) {
            const int64_t s0 = b * eb * P, s1 = std::min(ne, (b + 1) * eb) * P;
            int64_t cnt = 0;
            for (int64_t t = s0; t < s1 && dense; ++t) {
                const int32_t g = conn[(size_t)t];
                if (!seen[(size_t)g]) {
                    seen[(size_t)g] = 1;
                    if (g < next || g >= next + (s1 - s0)) dense = false;
                    cnt++;
                }
            }
            for (int64_t g = next; g < next + cnt && dense; ++g)
                if (g >= nn || !seen[(size_t)g]) dense = false;
            next += cnt;
        }
    }
    pl.dense = dense;
    // partial-sum slots: a contiguous run per open node, ascending node id
    std::vector<int64_t> base((size_t)nn, -1);
    {
        int64_t nopen = 0;
        for (int64_t g = 0; g < nn; ++g) nopen += nblk[(size_t)g] > 1;
        pl.open_gid.reserve((size_t)nopen);
        pl.open_base.reserve((size_t)nopen);
        pl.open_cnt.reserve((size_t)nopen);
    }
    for (int64_t g = 0; g < nn; ++g) {
        if (nblk[(size_t)g] > MAX_BLOCKS_PER_NODE) return "a node is touched by more than 255 element blocks";
        if (nblk[(size_t)g] > 1) {
            base[(size_t)g] = pl.npartial;
            pl.open_gid.push_back((int32_t)g);
            pl.open_base.push_back((int32_t)pl.npartial);
            pl.open_cnt.push_back(nblk[(size_t)g]);
            pl.npartial += nblk[(size_t)g];
        }
    }
    if (pl.npartial > INT32_MAX) return "too many partial sums";
    std::vector<int32_t> rec_of((size_t)nn, -1);
    for (size_t r = 0; r < rec_gid.size(); ++r)
        if (rec_gid[r] >= 0 && rec_of[(size_t)rec_gid[r]] < 0) rec_of[(size_t)rec_gid[r]] = (int32_t)r;
    pl.open_rec.resize(pl.open_gid.size());
    for (size_t k = 0; k < pl.open_gid.size(); ++k) pl.open_rec[k] = rec_of[(size_t)pl.open_gid[k]];

    const int UPH = (P + 1) / 2;
    pl.dev_order.resize((size_t)ne);
    pl.epos.assign((size_t)UPH * (size_t)ne, 0u);
    pl.hdr.assign((size_t)nb * HDR_INTS, 0);

    // pass 1 (sequential, linear): the entries of every block (owned nodes in
    // id order for DENSE, then the others by first appearance) and, per entry,
    // the rank of the block among the blocks that touch its node
    std::vector<int64_t> ent_ptr((size_t)nb + 1, 0), own_start_b((size_t)nb, 0), nown_b((size_t)nb, 0);
    std::vector<int32_t> ent_all;
    std::vector<uint8_t> rank_all;
    std::vector<int32_t> slot_block((size_t)pl.npartial, -1);  // block of each partial-sum slot
    ent_all.reserve((size_t)(nn + nn / 4));
    rank_all.reserve((size_t)(nn + nn / 4));
    {
        std::vector<int32_t> seen_rank((size_t)nn, 0);
        std::vector<int64_t> in_block((size_t)nn, -1);
        std::vector<uint8_t> touched((size_t)nn, 0);
        int64_t own_next = 0;
        for (int64_t b = 0; b < nb; ++b) {
            const int64_t e0 = b * eb, e1 = std::min(ne, e0 + eb);
            if (dense) {
                int64_t nown = 0;
                for (int64_t t = e0 * P; t < e1 * P; ++t) {
                    const int32_t g = conn[(size_t)t];
                    if (!touched[(size_t)g]) {
                        touched[(size_t)g] = 1;
                        nown++;
                    }
                }
                own_start_b[(size_t)b] = own_next;
                nown_b[(size_t)b] = nown;
                for (int64_t l = 0; l < nown; ++l) {
                    const int32_t g = (int32_t)(own_next + l);
                    in_block[(size_t)g] = b;
                    ent_all.push_back(g);
                }
                own_next += nown;
            }
            for (int64_t t = e0 * P; t < e1 * P; ++t) {
                const int32_t g = conn[(size_t)t];
                if (in_block[(size_t)g] != b) {
                    in_block[(size_t)g] = b;
                    ent_all.push_back(g);
                }
            }
            for (size_t k = (size_t)ent_ptr[(size_t)b]; k < ent_all.size(); ++k) {
                const int32_t g = ent_all[k];
                if (nblk[(size_t)g] > 1) slot_block[(size_t)(base[(size_t)g] + seen_rank[(size_t)g])] = (int32_t)b;
                rank_all.push_back((uint8_t)seen_rank[(size_t)g]++);
            }
            ent_ptr[(size_t)b + 1] = (int64_t)ent_all.size();
        }
    }

    // pass 2 (blocks in parallel): colouring, device order, local lists and
    // the packet body of each block, into per-block buffers; every write to
    // the shared outputs (hdr, dev_order, epos) touches the block's own part
    std::vector<std::vector<uint8_t>> bodies((size_t)nb);
    std::vector<std::vector<int32_t>> deps((size_t)nb);
    std::vector<int64_t> nclosed_b((size_t)nb, 0), nopen_b((size_t)nb, 0);
    std::vector<std::string> errs((size_t)nb);
    auto plan_block = [&](int64_t b) -> std::string {
        const int64_t e0 = b * eb, e1 = std::min(ne, e0 + eb);
        const int neb = (int)(e1 - e0);
        const int32_t* ent_gid = ent_all.data() + ent_ptr[(size_t)b];
        const uint8_t* rank = rank_all.data() + ent_ptr[(size_t)b];
        const int64_t nent = ent_ptr[(size_t)b + 1] - ent_ptr[(size_t)b];
        const int64_t own_start = own_start_b[(size_t)b], nown = nown_b[(size_t)b];
        const int64_t off = dense ? own_start % vec : 0;
        const int64_t ulen = dense ? align_up(off + nown, vec) : 0;
        const int64_t sulen = ulen + (nent - nown);
        const int64_t slen = dense ? ulen : nent;
        if (nent > 65535 || sulen > 65535) return "too many nodes in one element block";
        // entry of each slot: node ids sorted with their entry index
        std::vector<std::pair<int32_t, int32_t>> idx((size_t)nent);
        for (int64_t l = 0; l < nent; ++l) idx[(size_t)l] = {ent_gid[l], (int32_t)l};
        std::sort(idx.begin(), idx.end());
        std::vector<int32_t> slot_ent((size_t)neb * P);
        for (int64_t t = 0; t < (int64_t)neb * P; ++t) {
            const int32_t g = conn[(size_t)(e0 * P + t)];
            slot_ent[(size_t)t] = std::lower_bound(idx.begin(), idx.end(), std::make_pair(g, (int32_t)-1))->second;
        }
        // colouring of the block's conflict graph (elements sharing a node)
        // by DSatur: repeatedly colour the uncoloured element whose coloured
        // neighbours use the most distinct colours (ties: most neighbours,
        // then lowest index) with the smallest free colour
        std::vector<int32_t> elem_color((size_t)neb, -1);
        int ncolors = 0;
        {
            const int W = (neb + 63) / 64;
            std::vector<uint64_t> adj((size_t)neb * W, 0);
            // elements touching each entry (CSR, ascending element; an
            // element's slots are distinct nodes, so no element repeats)
            std::vector<int32_t> tptr((size_t)nent + 1, 0), tel((size_t)neb * P);
            for (int t = 0; t < neb * P; ++t) tptr[(size_t)slot_ent[(size_t)t] + 1]++;
            for (int64_t l = 0; l < nent; ++l) tptr[(size_t)l + 1] += tptr[(size_t)l];
            {
                std::vector<int32_t> fill(tptr.begin(), tptr.end() - 1);
                for (int t = 0; t < neb * P; ++t) tel[(size_t)fill[(size_t)slot_ent[(size_t)t]]++] = t / P;
            }
            for (int64_t l = 0; l < nent; ++l)
                for (int32_t x = tptr[(size_t)l]; x < tptr[(size_t)l + 1]; ++x)
                    for (int32_t y = x + 1; y < tptr[(size_t)l + 1]; ++y) {
                        const int ex = tel[(size_t)x], ey = tel[(size_t)y];
                        adj[(size_t)ex * W + ey / 64] |= 1ull << (ey % 64);
                        adj[(size_t)ey * W + ex / 64] |= 1ull << (ex % 64);
                    }
            std::vector<int> deg((size_t)neb, 0);
            for (int el = 0; el < neb; ++el)
                for (int w = 0; w < W; ++w) deg[(size_t)el] += __builtin_popcountll(adj[(size_t)el * W + w]);
            std::vector<uint32_t> sat((size_t)neb, 0);
            for (int it = 0; it < neb; ++it) {
                int best = -1, bs = -1, bd = -1;
                for (int el = 0; el < neb; ++el) {
                    if (elem_color[(size_t)el] >= 0) continue;
                    const int sv = __builtin_popcount(sat[(size_t)el]);
                    if (sv > bs || (sv == bs && deg[(size_t)el] > bd)) {
                        best = el;
                        bs = sv;
                        bd = deg[(size_t)el];
                    }
                }
                const uint32_t used = sat[(size_t)best];
                if (used == 0xFFFFFFFFu) return "more than 32 colours needed in one element block";
                int c = 0;
                while (used & (1u << c)) ++c;
                elem_color[(size_t)best] = c;
                ncolors = std::max(ncolors, c + 1);
                for (int w = 0; w < W; ++w) {
                    uint64_t bits = adj[(size_t)best * W + w];
                    while (bits) {
                        const int nb2 = w * 64 + __builtin_ctzll(bits);
                        bits &= bits - 1;
                        sat[(size_t)nb2] |= 1u << c;
                    }
                }
            }
        }
        // device order: stable sort by colour inside the block
        std::vector<int32_t> cstart((size_t)ncolors + 1, 0);
        for (int el = 0; el < neb; ++el) cstart[(size_t)elem_color[(size_t)el] + 1]++;
        for (int c = 0; c < ncolors; ++c) cstart[(size_t)c + 1] += cstart[(size_t)c];
        std::vector<int32_t> order_in_block((size_t)neb);
        {
            std::vector<int32_t> fill(cstart.begin(), cstart.end() - 1);
            for (int el = 0; el < neb; ++el) order_in_block[(size_t)fill[(size_t)elem_color[(size_t)el]]++] = el;
        }
        for (int i = 0; i < neb; ++i) pl.dev_order[(size_t)(e0 + i)] = e0 + order_in_block[(size_t)i];
        // open ranks in entry order
        std::vector<int32_t> orank_of((size_t)nent, -1);
        int64_t nopen = 0;
        for (int64_t l = 0; l < nent; ++l)
            if (nblk[(size_t)ent_gid[l]] > 1) orank_of[(size_t)l] = (int32_t)nopen++;
        if (nopen > 65535) return "too many open nodes in one element block";
        std::vector<int32_t> recs;
        int64_t nrc = 0, nro = 0;
        for (int64_t l = 0; l < nent; ++l) {
            const int32_t g = ent_gid[l];
            if (rec_of[(size_t)g] >= 0 && orank_of[(size_t)l] < 0) {
                recs.push_back(entry_pos((int)l, (int)nown, (int)off, (int)ulen));
                recs.push_back(rec_of[(size_t)g]);
                nrc++;
            }
        }
        for (int64_t l = 0; l < nent; ++l) {
            const int32_t g = ent_gid[l];
            if (rec_of[(size_t)g] >= 0 && orank_of[(size_t)l] >= 0 && rank[l] == 0) {
                recs.push_back(entry_pos((int)l, (int)nown, (int)off, (int)ulen));
                recs.push_back(rec_of[(size_t)g]);
                nro++;
            }
        }
        const Offsets L = offsets((int)sulen, (int)ulen, (int)nopen, ncolors, (int)(nrc + nro));
        std::vector<uint8_t>& body = bodies[(size_t)b];
        body.assign((size_t)L.bytes, 0);
        uint8_t* pk = body.data();
        uint32_t* cmask = reinterpret_cast<uint32_t*>(pk + L.cmask);
        int32_t* egid = reinterpret_cast<int32_t*>(pk + L.egid);
        int32_t* obase = reinterpret_cast<int32_t*>(pk + L.obase);
        uint16_t* opos = reinterpret_cast<uint16_t*>(pk + L.opos);
        uint8_t* ocnt = pk + L.ocnt;
        uint8_t* orank = pk + L.orank;
        uint16_t* pcs = reinterpret_cast<uint16_t*>(pk + L.cstart);
        int32_t* prec = reinterpret_cast<int32_t*>(pk + L.recs);
        int64_t nclosed = 0;
        for (int64_t l = 0; l < nent; ++l) {
            const int32_t g = ent_gid[l];
            const int32_t o = orank_of[(size_t)l];
            const int pos = entry_pos((int)l, (int)nown, (int)off, (int)ulen);
            if (o < 0) {
                cmask[pos >> 5] |= 1u << (pos & 31);
                nclosed++;
            } else {
                obase[o] = (int32_t)base[(size_t)g];
                opos[o] = (uint16_t)pos;
                ocnt[o] = (uint8_t)nblk[(size_t)g];
                orank[o] = rank[l];
            }
            if (l >= nown) egid[pos - ulen] = g;
        }
        for (int c = 0; c <= ncolors; ++c) pcs[c] = (uint16_t)cstart[(size_t)c];
        std::copy(recs.begin(), recs.end(), prec);
        for (int i = 0; i < neb; ++i) {
            const int el = order_in_block[(size_t)i];
            for (int q = 0; q < P; ++q) {
                const int l = slot_ent[(size_t)(el * P + q)];
                const uint32_t pos = (uint32_t)entry_pos(l, (int)nown, (int)off, (int)ulen);
                pl.epos[(size_t)(q / 2) * (size_t)ne + (size_t)(e0 + i)] |= pos << (16 * (q & 1));
            }
        }
        int32_t* h = &pl.hdr[(size_t)b * HDR_INTS];
        h[H_NENT] = (int32_t)nent;
        h[H_NOWN] = (int32_t)nown;
        h[H_OWN_START] = (int32_t)own_start;
        h[H_NOPEN] = (int32_t)nopen;
        h[H_ULEN] = (int32_t)ulen;
        h[H_SLEN] = (int32_t)slen;
        h[H_SULEN] = (int32_t)sulen;
        h[H_NCOLORS] = ncolors;
        h[H_NREC_CLOSED] = (int32_t)nrc;
        h[H_NREC_OPEN] = (int32_t)nro;
        nclosed_b[(size_t)b] = nclosed;
        nopen_b[(size_t)b] = nopen;
        std::vector<int32_t>& dl = deps[(size_t)b];
        dl.push_back((int32_t)b);
        for (int64_t l = 0; l < nent; ++l) {
            const int32_t g = ent_gid[l];
            if (nblk[(size_t)g] > 1)
                for (int r = 0; r < nblk[(size_t)g]; ++r) dl.push_back(slot_block[(size_t)(base[(size_t)g] + r)]);
        }
        std::sort(dl.begin(), dl.end());
        dl.erase(std::unique(dl.begin(), dl.end()), dl.end());
        return "";
    };
    {
        std::atomic<int64_t> next(0);
        const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
        const unsigned nthr = (unsigned)std::min<int64_t>(hw, std::max<int64_t>(1, nb / 8));
        auto work = [&]() {
            for (int64_t b = next++; b < nb; b = next++) errs[(size_t)b] = plan_block(b);
        };
        std::vector<std::thread> pool;
        for (unsigned t = 1; t < nthr; ++t) pool.emplace_back(work);
        work();
        for (auto& t : pool) t.join();
    }
    for (int64_t b = 0; b < nb; ++b)
        if (!errs[(size_t)b].empty()) return errs[(size_t)b];

    // pass 3: the packets block after block, and the plan's maxima
    size_t total = 0;
    for (const auto& body : bodies) total += body.size();
    pl.packet.resize(total);
    size_t start = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const auto& body = bodies[(size_t)b];
        std::memcpy(pl.packet.data() + start, body.data(), body.size());
        int32_t* h = &pl.hdr[(size_t)b * HDR_INTS];
        h[H_START] = (int32_t)(start / 16);
        start += body.size();
        pl.max_entries = std::max<int>(pl.max_entries, h[H_NENT]);
        pl.max_sulen = std::max<int>(pl.max_sulen, h[H_SULEN]);
        pl.max_slen = std::max<int>(pl.max_slen, h[H_SLEN]);
        pl.max_packet = std::max<int>(pl.max_packet, (int)body.size());
        pl.max_colors = std::max(pl.max_colors, h[H_NCOLORS]);
        pl.nent_total += h[H_NENT];
        pl.nopen_entries += nopen_b[(size_t)b];
        pl.nclosed_total += nclosed_b[(size_t)b];
        std::vector<uint8_t>().swap(bodies[(size_t)b]);
    }
    if ((int64_t)pl.packet.size() / 16 > INT32_MAX) return "packet array too large";
    pl.dep_ptr.assign((size_t)nb + 1, 0);
    for (int64_t b = 0; b < nb; ++b) {
        pl.dep_ptr[(size_t)b + 1] = pl.dep_ptr[(size_t)b] + (int32_t)deps[(size_t)b].size();
        pl.max_deps = std::max(pl.max_deps, (int)deps[(size_t)b].size());
    }
    pl.dep.reserve((size_t)pl.dep_ptr[(size_t)nb]);
    for (auto& dl : deps) pl.dep.insert(pl.dep.end(), dl.begin(), dl.end());
    return "";
}

std::string check_block_plan(const BlockPlan& pl, const std::vector<int32_t>& conn, int vec) {
    using namespace semplan;
    const int P = pl.P;
    const int64_t ne = pl.ne, nn = pl.nn;
    auto fail = [](int64_t b, const std::string& what) { return "block " + std::to_string(b) + ": " + what; };
    // the device order permutes elements inside their blocks only
    {
        std::vector<uint8_t> hit((size_t)ne, 0);
        for (int64_t i = 0; i < ne; ++i) {
            const int64_t e = pl.dev_order[(size_t)i];
            if (e < 0 || e >= ne || hit[(size_t)e] || e / pl.eb != i / pl.eb) return "device order is not a per-block permutation";
            hit[(size_t)e] = 1;
        }
    }
    std::vector<double> u((size_t)nn), out((size_t)nn, std::nan("")), ref((size_t)nn, 0.0);
    for (int64_t g = 0; g < nn; ++g) u[(size_t)g] = (double)((g * 37) % 1001);
    for (int64_t s = 0; s < ne * P; ++s) {
        const int64_t e = s / P;
        ref[(size_t)conn[(size_t)s]] += u[(size_t)conn[(size_t)s]] + (double)((e % 7) * (s % P + 1));
    }
    std::vector<double> part((size_t)std::max<int64_t>(pl.npartial, 1), std::nan(""));
    std::vector<double> su, acc;
    std::vector<int64_t> stamp;
    int64_t phase = 0;
    for (int64_t b = 0; b < pl.nblocks; ++b) {
        const int32_t* h = &pl.hdr[(size_t)b * HDR_INTS];
        const int64_t e0 = b * pl.eb;
        const int neb = (int)std::min<int64_t>(pl.eb, ne - e0);
        const int nent = h[H_NENT], nown = h[H_NOWN], own_start = h[H_OWN_START], nopen = h[H_NOPEN];
        const int ulen = h[H_ULEN], slen = h[H_SLEN], sulen = h[H_SULEN], ncolors = h[H_NCOLORS];
        const int nrc = h[H_NREC_CLOSED], nro = h[H_NREC_OPEN];
        const int off = pl.dense ? own_start % vec : 0;
        const int64_t abase = (int64_t)own_start - off;
        if (sulen != ulen + nent - nown) return fail(b, "position count mismatch");
        if (sulen > pl.max_sulen || slen > pl.max_slen || nent > pl.max_entries) return fail(b, "size above maximum");
        if (slen > sulen) return fail(b, "staged range beyond positions");
        if (pl.dense && (ulen % vec != 0 || abase % vec != 0 || slen != ulen)) return fail(b, "owned range misaligned");
        if (ncolors < 1 || ncolors > MAX_COLORS) return fail(b, "colour count");
        const Offsets L = offsets(sulen, ulen, nopen, ncolors, nrc + nro);
        const int64_t start = (int64_t)h[H_START] * 16;
        if (L.bytes > pl.max_packet || start + L.bytes > (int64_t)pl.packet.size()) return fail(b, "packet bounds");
        const uint8_t* pk = pl.packet.data() + start;
        const uint32_t* cmask = reinterpret_cast<const uint32_t*>(pk + L.cmask);
        const int32_t* egid = reinterpret_cast<const int32_t*>(pk + L.egid);
        const int32_t* obase = reinterpret_cast<const int32_t*>(pk + L.obase);
        const uint16_t* opos = reinterpret_cast<const uint16_t*>(pk + L.opos);
        const uint8_t* ocnt = pk + L.ocnt;
        const uint8_t* orank = pk + L.orank;
        const uint16_t* cstart = reinterpret_cast<const uint16_t*>(pk + L.cstart);
        const int32_t* recs = reinterpret_cast<const int32_t*>(pk + L.recs);
        auto gid_at = [&](int p) -> int64_t { return p < ulen ? abase + p : (int64_t)egid[p - ulen]; };
        auto closed = [&](int p) { return (cmask[p >> 5] >> (p & 31)) & 1u; };
        // node values: owned range as aligned vectors, then the other positions
        su.assign((size_t)sulen, std::nan(""));
        for (int p = 0; p < ulen; ++p) {
            const int64_t g = abase + p;
            if (g >= 0 && g < nn) su[(size_t)p] = u[(size_t)g];
        }
        for (int p = ulen; p < sulen; ++p) {
            const int64_t g = gid_at(p);
            if (g < 0 || g >= nn) return fail(b, "node id out of range");
            su[(size_t)p] = u[(size_t)g];
        }
        // element residuals through epos, scattered colour by colour
        if (cstart[0] != 0 || cstart[ncolors] != neb) return fail(b, "colour ranges do not cover the block");
        acc.assign((size_t)sulen, 0.0);
        stamp.assign((size_t)sulen, -1);
        for (int c = 0; c < ncolors; ++c) {
            if (cstart[c + 1] < cstart[c]) return fail(b, "colour ranges not monotone");
            ++phase;
            for (int i = cstart[c]; i < cstart[c + 1]; ++i) {
                const int64_t e = pl.dev_order[(size_t)(e0 + i)];
                for (int q = 0; q < P; ++q) {
                    const uint32_t w = pl.epos[(size_t)(q / 2) * (size_t)ne + (size_t)(e0 + i)];
                    const int pos = (int)((w >> (16 * (q & 1))) & 0xFFFF);
                    if (pos >= sulen) return fail(b, "epos beyond node values");
                    const int64_t g = conn[(size_t)(e * P + q)];
                    if (su[(size_t)pos] != u[(size_t)g] || gid_at(pos) != g) return fail(b, "slot reads another node's value");
                    if (stamp[(size_t)pos] == phase) return fail(b, "two elements of one colour share a node");
                    stamp[(size_t)pos] = phase;
                    acc[(size_t)pos] += su[(size_t)pos] + (double)((e % 7) * (q + 1));
                }
            }
        }
        // closed positions finish their node, open entries leave a partial
        int nclosed_seen = 0;
        for (int p = 0; p < sulen; ++p) {
            if (!closed(p)) continue;
            if (p >= slen) return fail(b, "closed entry outside staged state");
            if (p < ulen && (p < off || p >= off + nown)) return fail(b, "closed bit on a padding position");
            const int64_t g = gid_at(p);
            if (!std::isnan(out[(size_t)g])) return fail(b, "node finished twice");
            out[(size_t)g] = acc[(size_t)p];
            nclosed_seen++;
        }
        for (int o = 0; o < nopen; ++o) {
            const int p = opos[o];
            if (p >= sulen || closed(p)) return fail(b, "open position");
            if (p < ulen && (p < off || p >= off + nown)) return fail(b, "open entry on a padding position");
            if (orank[o] >= ocnt[o]) return fail(b, "open rank beyond its node's block count");
            if (orank[o] == 0 && p >= slen) return fail(b, "owner's open entry outside staged state");
            const int64_t pi = (int64_t)obase[o] + orank[o];
            if (pi < 0 || pi >= pl.npartial) return fail(b, "partial index out of range");
            if (!std::isnan(part[(size_t)pi])) return fail(b, "partial slot written twice");
            part[(size_t)pi] = acc[(size_t)p];
        }
        if (nclosed_seen + nopen != nent) return fail(b, "closed + open != entries");
        for (int k = 0; k < nrc + nro; ++k) {
            const int p = recs[2 * k];
            if (p >= slen) return fail(b, "receiver record outside staged state");
            if (k < nrc && !closed(p)) return fail(b, "closed receiver record on an open entry");
            if (k >= nrc && closed(p)) return fail(b, "open receiver record on a closed entry");
        }
    }
    for (size_t k = 0; k < pl.open_gid.size(); ++k) {
        double s = 0.0;
        for (int t = 0; t < pl.open_cnt[k]; ++t) {
            const double v = part[(size_t)(pl.open_base[k] + t)];
            if (std::isnan(v)) return "open node " + std::to_string(pl.open_gid[k]) + ": missing partial";
            s += v;
        }
        if (!std::isnan(out[(size_t)pl.open_gid[k]])) return "open node also finished by a block";
        out[(size_t)pl.open_gid[k]] = s;
    }
    for (int64_t g = 0; g < nn; ++g)
        if (out[(size_t)g] != ref[(size_t)g]) return "node " + std::to_string(g) + ": assembled value differs";
    // neighbour lists: exactly the blocks sharing a node with the block
    // (itself included), ascending, from the connectivity directly
    {
        const int64_t nbk = pl.nblocks;
        if ((int64_t)pl.dep_ptr.size() != nbk + 1 || pl.dep_ptr[0] != 0 ||
            (int64_t)pl.dep.size() != (int64_t)pl.dep_ptr[(size_t)nbk])
            return "neighbour lists: bad sizes";
        std::vector<std::vector<int32_t>> node_blocks((size_t)nn);
        for (int64_t t = 0; t < pl.ne * pl.P; ++t) {
            auto& v = node_blocks[(size_t)conn[(size_t)t]];
            const int32_t b = (int32_t)(t / pl.P / pl.eb);
            if (std::find(v.begin(), v.end(), b) == v.end()) v.push_back(b);
        }
        std::vector<std::vector<int32_t>> want((size_t)nbk);
        for (const auto& v : node_blocks)
            for (int32_t x : v)
                for (int32_t y : v) want[(size_t)x].push_back(y);
        for (int64_t b = 0; b < nbk; ++b) {
            auto& w = want[(size_t)b];
            w.push_back((int32_t)b);
            std::sort(w.begin(), w.end());
            w.erase(std::unique(w.begin(), w.end()), w.end());
            const std::vector<int32_t> got(pl.dep.begin() + pl.dep_ptr[(size_t)b], pl.dep.begin() + pl.dep_ptr[(size_t)b + 1]);
            if (got != w) return "block " + std::to_string(b) + ": neighbour list differs";
        }
    }
    return "";
}


std::vector<int32_t> block_levels(const int32_t* dep_ptr, const int32_t* dep, int64_t nb) {
    std::vector<int32_t> lev((size_t)nb, -1), first((size_t)nb, -1), queue;
    queue.reserve((size_t)nb);
    // breadth-first sweep from root over one connected part; returns the
    // block reached last at the largest distance (the lowest id among those)
    auto sweep = [&](int32_t root, std::vector<int32_t>& L) {
        queue.clear();
        queue.push_back(root);
        L[(size_t)root] = 0;
        int32_t far = root;
        for (size_t h = 0; h < queue.size(); ++h) {
            const int32_t x = queue[h];
            if (L[(size_t)x] > L[(size_t)far] || (L[(size_t)x] == L[(size_t)far] && x < far)) far = x;
            for (int32_t t = dep_ptr[x]; t < dep_ptr[x + 1]; ++t) {
                const int32_t y = dep[t];
                if (L[(size_t)y] < 0) {
                    L[(size_t)y] = L[(size_t)x] + 1;
                    queue.push_back(y);
                }
            }
        }
        return far;
    };
    for (int64_t r = 0; r < nb; ++r)
        if (lev[(size_t)r] < 0) sweep(sweep((int32_t)r, first), lev);
    return lev;
}

int auto_window(const std::vector<int32_t>& levels, int64_t target_units) {
    int32_t top = 0;
    for (int32_t l : levels) top = std::max(top, l);
    const double per_level = (double)levels.size() / (double)(top + 1);
    const double w = std::floor((double)target_units / std::max(1.0, per_level) + 0.5);
    return (int)std::max(1.0, std::min(w, (double)(top + 1)));
}

std::string stream_schedule(const int32_t* dep_ptr, const int32_t* dep, int64_t nb, int T, int W,
                            std::vector<uint32_t>& sched, std::vector<int32_t>* levels_out) {
    if (T < 1 || T > kSchedMaxSteps) return "band of steps outside 1.." + std::to_string(kSchedMaxSteps);
    if (W < 1) return "window below one level";
    if (nb < 1 || nb >= ((int64_t)1 << kSchedShift)) return "block count outside the schedule's range";
    const std::vector<int32_t> lev = block_levels(dep_ptr, dep, nb);
    int32_t top = 0;
    for (int32_t l : lev) top = std::max(top, l);
    // blocks grouped by level, ascending id within a level
    std::vector<int64_t> lptr((size_t)top + 2, 0);
    for (int32_t l : lev) ++lptr[(size_t)l + 1];
    for (int32_t l = 0; l <= top; ++l) lptr[(size_t)l + 1] += lptr[(size_t)l];
    std::vector<int32_t> by_level((size_t)nb);
    {
        std::vector<int64_t> fill(lptr.begin(), lptr.end() - 1);
        for (int64_t b = 0; b < nb; ++b) by_level[(size_t)fill[(size_t)lev[(size_t)b]]++] = (int32_t)b;
    }
    sched.clear();
    sched.reserve((size_t)(T * nb));
    const int64_t tiles = (int64_t)(top + T - 1) / W + 1;
    for (int64_t t = 0; t < tiles; ++t)
        for (int j = 0; j < T; ++j) {
            // levels l with floor((l + j) / W) == t
            const int64_t lo = std::max<int64_t>(0, t * W - j), hi = std::min<int64_t>(top, (t + 1) * W - j - 1);
            for (int64_t l = lo; l <= hi; ++l)
                for (int64_t k = lptr[(size_t)l]; k < lptr[(size_t)l + 1]; ++k)
                    sched.push_back(((uint32_t)j << kSchedShift) | (uint32_t)by_level[(size_t)k]);
        }
    if ((int64_t)sched.size() != T * nb) return "schedule does not cover the band";
    if (levels_out) *levels_out = lev;
    return "";
}

std::string check_stream_schedule(const int32_t* dep_ptr, const int32_t* dep, int64_t nb, int T,
                                  const std::vector<uint32_t>& sched) {
    if ((int64_t)sched.size() != T * nb) return "schedule length differs from steps x blocks";
    std::vector<int64_t> pos((size_t)(T * nb), -1);
    const uint32_t mask = (1u << kSchedShift) - 1u;
    for (size_t k = 0; k < sched.size(); ++k) {
        const int64_t j = sched[k] >> kSchedShift, b = sched[k] & mask;
        if (j >= T || b >= nb) return "entry " + std::to_string(k) + " outside the band";
        int64_t& p = pos[(size_t)(j * nb + b)];
        if (p >= 0) return "unit (" + std::to_string(j) + ", " + std::to_string(b) + ") listed twice";
        p = (int64_t)k;
    }
    for (int64_t j = 1; j < T; ++j)
        for (int64_t b = 0; b < nb; ++b)
            for (int32_t t = dep_ptr[b]; t < dep_ptr[b + 1]; ++t)
                if (pos[(size_t)((j - 1) * nb + dep[t])] > pos[(size_t)(j * nb + b)])
                    return "unit (" + std::to_string(j) + ", " + std::to_string(b) + ") precedes step " +
                           std::to_string(j - 1) + " of block " + std::to_string(dep[t]);
    return "";
}

}  // namespace semhost
