// Host-side plan construction: FP64 geometry and GCF taps (paper Sec. 2, Eq. 1
// bracket: W_e^*(r_j - r_e) evaluated at the grid points r_j around each
// element), the inverse cell -> (element, weight) lists used for atomic-free
// gridding, and the transform twiddles.  Pure host code, no CUDA launches.
#include <math.h>

#include <algorithm>
#include <cstdio>

#include "epic_internal.h"

namespace epic {

static const double kC0 = 299792458.0;
static const double kPi = 3.14159265358979323846;

// Element cell coordinates u = (x - xbar)/Delta + N/2 (centroid at the grid
// centre), first tap per axis (odd K: nearest cell, ties up, minus (K-1)/2; even
// K: floor(u) - K/2 + 1), and conj(W(j - u)) for each tap.  The fftshift of the
// output is folded in: every tap weight at cell (jx, jy) carries (-1)^(jx+jy),
// which moves Fourier index k to k + N/2 so that the transform writes the
// zero direction at image index N/2 directly.
epic_status build_geometry(epic_plan_s* p, std::string* err)
{
    const int A = p->A, C = p->C, N = p->N, K = p->K;
    double xbar = 0.0, ybar = 0.0;
    for (int e = 0; e < A; ++e) {
        xbar += p->pos[2 * e];
        ybar += p->pos[2 * e + 1];
    }
    xbar /= A;
    ybar /= A;
    p->box.assign(C, Box{0, 0, 0, 0});
    p->first_x.assign((size_t)C * A, 0);
    p->first_y.assign((size_t)C * A, 0);
    p->w_re.assign((size_t)C * A * K * K, 0.0);
    p->w_im.assign((size_t)C * A * K * K, 0.0);
    p->box_max_x = p->box_max_y = 0;
    for (int c = 0; c < C; ++c) {
        const double f = p->freq[c];
        const double lam = kC0 / f;
        const double delta = p->cell.empty() ? 0.5 * lam : p->cell[c];
        if (!(delta > 0.0) || !std::isfinite(delta)) {
            *err = "cell spacing must be positive and finite";
            return EPIC_ERR_INVALID_ARG;
        }
        double sig = p->gcf.sigma_cells;
        if (p->gcf.freq_scaled) sig = p->gcf.sigma_cells * f / p->gcf.f_ref_hz;
        int xmin = N, xmax = -1, ymin = N, ymax = -1;
        for (int e = 0; e < A; ++e) {
            const double u = (p->pos[2 * e] - xbar) / delta + 0.5 * N;
            const double v = (p->pos[2 * e + 1] - ybar) / delta + 0.5 * N;
            if (!std::isfinite(u) || !std::isfinite(v) || fabs(u) > 1e9 || fabs(v) > 1e9) {
                *err = "element position maps outside any grid";
                return EPIC_ERR_GRID_OVERFLOW;
            }
            long fx, fy;
            if (K % 2 == 1) {
                fx = (long)floor(u + 0.5) - (K - 1) / 2;
                fy = (long)floor(v + 0.5) - (K - 1) / 2;
            } else {
                fx = (long)floor(u) - K / 2 + 1;
                fy = (long)floor(v) - K / 2 + 1;
            }
            if (fx < 0 || fy < 0 || fx + K - 1 >= N || fy + K - 1 >= N) {
                char buf[160];
                snprintf(buf, sizeof buf, "GCF footprint of element %d leaves the %dx%d grid in channel %d", e, N,
                         N, c);
                *err = buf;
                return EPIC_ERR_GRID_OVERFLOW;
            }
            p->first_x[(size_t)c * A + e] = (int)fx;
            p->first_y[(size_t)c * A + e] = (int)fy;
            xmin = std::min(xmin, (int)fx);
            xmax = std::max(xmax, (int)fx + K - 1);
            ymin = std::min(ymin, (int)fy);
            ymax = std::max(ymax, (int)fy + K - 1);
            for (int ty = 0; ty < K; ++ty) {
                for (int tx = 0; tx < K; ++tx) {
                    const int jx = (int)fx + tx, jy = (int)fy + ty;
                    const double dx = (double)jx - u, dy = (double)jy - v;
                    double wr, wi;
                    if (p->gcf.kind == EPIC_GCF_GAUSSIAN) {
                        wr = exp(-(dx * dx + dy * dy) / (2.0 * sig * sig));
                        wi = 0.0;
                    } else {
                        const int os = p->gcf.oversample;
                        const int side = K * os + 1;
                        int ix = (int)floor((dx + 0.5 * K) * os + 0.5);
                        int iy = (int)floor((dy + 0.5 * K) * os + 0.5);
                        ix = std::min(std::max(ix, 0), side - 1);
                        iy = std::min(std::max(iy, 0), side - 1);
                        wr = p->table[2 * ((size_t)iy * side + ix)];
                        wi = -(double)p->table[2 * ((size_t)iy * side + ix) + 1];  // W*
                    }
                    const double sgn = ((jx + jy) & 1) ? -1.0 : 1.0;
                    const size_t o = (((size_t)c * A + e) * K + ty) * K + tx;
                    p->w_re[o] = sgn * wr;
                    p->w_im[o] = sgn * wi;
                }
            }
        }
        // Occupied box, widths padded (cells beyond the footprints stay empty): x to a
        // multiple of 8, y to 8 (two pols) or 16 (one pol), as the tensor-core path needs
        // (MMA K steps of 16 halves over re|im of x, N = pols x rows a multiple of 16).
        const int padx = 8, pady = p->P == 2 ? 8 : 16;
        const int nx = (xmax - xmin + 1 + padx - 1) / padx * padx;
        const int ny = (ymax - ymin + 1 + pady - 1) / pady * pady;
        p->box[c] = Box{xmin, ymin, nx, ny};
        p->box_max_x = std::max(p->box_max_x, nx);
        p->box_max_y = std::max(p->box_max_y, ny);
    }
    p->n_contrib = (size_t)C * A * K * K;
    return EPIC_OK;
}

// Inverse of the footprints: for every cell of channel c's occupied box (row
// major, r = (y - y0) * nx + (x - x0)) the list of (element, weight) that lands
// there, in element order.  Gridding then gathers per cell with no conflicts.
void build_csr(const epic_plan_s* p, std::vector<int>& cell_off, std::vector<int>& cell_ptr,
               std::vector<int>& contrib_e, std::vector<float2>& contrib_w)
{
    const int A = p->A, C = p->C, K = p->K;
    cell_off.assign(C + 1, 0);
    size_t ncell = 0;
    for (int c = 0; c < C; ++c) {
        cell_off[c] = (int)ncell;
        ncell += (size_t)p->box[c].nx * p->box[c].ny + 1;
    }
    cell_off[C] = (int)ncell;
    cell_ptr.assign(ncell, 0);
    contrib_e.assign(p->n_contrib, 0);
    contrib_w.assign(p->n_contrib, make_float2(0.f, 0.f));
    size_t base = 0;
    std::vector<int> fill;
    for (int c = 0; c < C; ++c) {
        const Box b = p->box[c];
        const int nb = b.nx * b.ny;
        int* ptr = &cell_ptr[cell_off[c]];
        std::vector<int> cnt(nb + 1, 0);
        for (int e = 0; e < A; ++e) {
            const int fx = p->first_x[(size_t)c * A + e] - b.x0, fy = p->first_y[(size_t)c * A + e] - b.y0;
            for (int ty = 0; ty < K; ++ty)
                for (int tx = 0; tx < K; ++tx) cnt[(fy + ty) * b.nx + fx + tx + 1]++;
        }
        ptr[0] = (int)base;
        for (int r = 0; r < nb; ++r) ptr[r + 1] = ptr[r] + cnt[r + 1];
        fill.assign(nb, 0);
        for (int e = 0; e < A; ++e) {
            const int fx = p->first_x[(size_t)c * A + e] - b.x0, fy = p->first_y[(size_t)c * A + e] - b.y0;
            for (int ty = 0; ty < K; ++ty)
                for (int tx = 0; tx < K; ++tx) {
                    const int r = (fy + ty) * b.nx + fx + tx;
                    const size_t dst = (size_t)ptr[r] + fill[r]++;
                    const size_t o = (((size_t)c * A + e) * K + ty) * K + tx;
                    contrib_e[dst] = e;
                    contrib_w[dst] = make_float2((float)p->w_re[o], (float)p->w_im[o]);
                }
        }
        base += (size_t)A * K * K;
    }
}

// exp(+2 pi i m / N) for m in [0, N/2), from host FP64 libm.
void build_twiddles(int N, std::vector<float2>& tw)
{
    tw.resize(N / 2);
    for (int m = 0; m < N / 2; ++m) {
        const double a = 2.0 * kPi * (double)m / (double)N;
        tw[m] = make_float2((float)cos(a), (float)sin(a));
    }
}

// Interleaves the (element, payload) entries of one warp's tasks for the balanced
// gridding kernel: entry k of lane l goes to out[32 k + l], every lane padded to nmax
// entries with payload 0 (which the caller reads as zero weights).  A task's sums do
// not depend on the order of its entries beyond FP32 rounding, so the order is chosen
// for the shared-memory gather:
// at step k the lanes of a warp read the 16-byte voltages of their k-th elements,
// and 8 lanes that ask for different elements in the same 16-byte bank quad
// (element mod 8) serialise.  Per step and per group of 8 lanes, lanes that must take
// an entry now come first, then those with the fewest distinct quads left; each
// takes an element another lane already reads (a broadcast), else one on an unused
// quad (the quad most in demand among the group's remaining entries), else, if it
// has slack, a padding entry on an element already read.
void order_warp_entries(const std::vector<std::vector<int2>>& cells, int nmax, int2* out)
{
    const int members = (int)cells.size();
    std::vector<std::vector<int2>> rem(cells);
    for (int k = 0; k < nmax; ++k) {
        const int left = nmax - k;
        for (int q0 = 0; q0 < 32; q0 += 8) {
            int demand[8] = {0, 0, 0, 0, 0, 0, 0, 0}, used[8], lanes[8], key[8], nl = 0, first = -1;
            bool pad[8] = {false, false, false, false, false, false, false, false};
            for (int q = 0; q < 8; ++q) used[q] = -1;
            for (int l = q0; l < q0 + 8 && l < members; ++l) {
                unsigned quads = 0;
                for (const int2& en : rem[l]) {
                    demand[en.x & 7]++;
                    quads |= 1u << (en.x & 7);
                }
                int nq = 0;
                for (int q = 0; q < 8; ++q) nq += (quads >> q) & 1u;
                key[nl] = ((int)rem[l].size() == left ? 0 : 16) + (rem[l].empty() ? 15 : nq);
                lanes[nl++] = l;
            }
            for (int i = 1; i < nl; ++i)  // stable insertion sort by key
                for (int j = i; j > 0 && key[j - 1] > key[j]; --j) {
                    std::swap(key[j - 1], key[j]);
                    std::swap(lanes[j - 1], lanes[j]);
                }
            for (int i = 0; i < nl; ++i) {
                std::vector<int2>& r = rem[lanes[i]];
                int pick = -1;
                for (int j = 0; j < (int)r.size() && pick < 0; ++j)
                    if (used[r[j].x & 7] == r[j].x) pick = j;
                if (pick < 0) {
                    int best = -1;
                    for (int j = 0; j < (int)r.size(); ++j) {
                        const int q = r[j].x & 7;
                        if (used[q] < 0 && demand[q] > best) {
                            best = demand[q];
                            pick = j;
                        }
                    }
                }
                if (pick < 0) {
                    if ((int)r.size() < left) {  // empty, or slack left: pad this step
                        pad[i] = true;
                        continue;
                    }
                    pick = 0;
                }
                const int2 en = r[pick];
                if (used[en.x & 7] < 0) {
                    used[en.x & 7] = en.x;
                    if (first < 0) first = en.x;
                }
                out[32 * k + lanes[i]] = en;
                r.erase(r.begin() + pick);
            }
            const int2 zero = make_int2(first < 0 ? 0 : first, 0);
            for (int i = 0; i < nl; ++i)
                if (pad[i]) out[32 * k + lanes[i]] = zero;
            for (int l = std::max(q0, members); l < q0 + 8; ++l) out[32 * k + l] = zero;
        }
    }
}

}  // namespace epic
