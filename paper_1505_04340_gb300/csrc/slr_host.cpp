// Host-side setup of the SLR preconditioner: everything that runs once per
// matrix before the device takes over (Sections 2.1, 3.1 and 5.2 of Li, Xi &
// Saad, arXiv 1505.04340).
//
//  * host_validate_csr  - CSR structure, symmetry and partition checks
//  * host_dd_order      - interface detection of a vertex-based partition and
//                         the global ordering [u_1..u_p, y_1..y_p] (Eqs. 2.2-2.3)
//  * host_split_blocks  - P A P^T, E, E^T and C in CSR
//  * host_band_factor   - exact banded Cholesky of every B_i (Section 5.2),
//                         repacked plane by plane with inverted diagonal blocks
//  * host_c_factor      - exact Cholesky C = L L^T (Eq. 3.1) in a nested
//                         dissection order, supernodal, kept as inverted diagonal
//                         blocks L_JJ^{-1} and panels M_J = L[R_J, J] L_JJ^{-1},
//                         with a level schedule for the device solves
//  * host_c_top         - explicit inverse of the factor's top levels (partitioned
//                         inverse) for one-step solves of that zone
//  * host_tridiag_eig   - eigenpairs of the Lanczos tridiagonal (Section 5.1), implicit QL
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "slr_internal.h"

namespace slr {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

double splitmix_pm1(uint64_t seed, uint64_t i) {
    // SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator.
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    return 2.0 * u - 1.0;
}

// ------------------------------------------------------------------ checks

slr_status host_validate_csr(int32_t n, const int32_t* rowptr, const int32_t* colind,
                             const double* val, int32_t nparts, const int32_t* part) {
    if (n < 0 || (n > 0 && (!rowptr || !part)) || nparts < 1) {
        set_error("invalid sizes or NULL pointers");
        return SLR_ERR_INVALID_ARG;
    }
    if (n == 0) return SLR_OK;
    if (rowptr[0] != 0) { set_error("rowptr[0] != 0"); return SLR_ERR_INVALID_ARG; }
    for (int32_t i = 0; i < n; ++i)
        if (rowptr[i + 1] < rowptr[i]) { set_error("rowptr not monotone"); return SLR_ERR_INVALID_ARG; }
    int64_t nnz = rowptr[n];
    if (nnz > 0 && (!colind || !val)) { set_error("NULL colind/val"); return SLR_ERR_INVALID_ARG; }
    for (int32_t i = 0; i < n; ++i)
        if (part[i] < -1 || part[i] >= nparts) {   // -1: a vertex-separator node
            set_error("part[" + std::to_string(i) + "] out of range");
            return SLR_ERR_INVALID_ARG;
        }
    // per-row sorted copy of the columns to check duplicates and symmetry
    std::vector<std::pair<int32_t, double>> row;
    std::vector<int32_t> sc(nnz);
    std::vector<double> sv(nnz);
    for (int32_t i = 0; i < n; ++i) {
        row.clear();
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            if (colind[q] < 0 || colind[q] >= n) {
                set_error("column index out of range in row " + std::to_string(i));
                return SLR_ERR_INVALID_ARG;
            }
            row.emplace_back(colind[q], val[q]);
        }
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                      return a.first < b.first;
                  });
        for (size_t t = 0; t < row.size(); ++t) {
            if (t && row[t].first == row[t - 1].first) {
                set_error("duplicate entry in row " + std::to_string(i));
                return SLR_ERR_INVALID_ARG;
            }
            sc[rowptr[i] + t] = row[t].first;
            sv[rowptr[i] + t] = row[t].second;
        }
    }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            int32_t j = sc[q];
            const int32_t* b = sc.data() + rowptr[j];
            const int32_t* e = sc.data() + rowptr[j + 1];
            const int32_t* f = std::lower_bound(b, e, i);
            if (f == e || *f != i) {
                set_error("pattern not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")");
                return SLR_ERR_INVALID_ARG;
            }
            double a = sv[q], c = sv[f - sc.data()];
            if (std::fabs(a - c) > 1e-12 * std::max(std::fabs(a), std::fabs(c))) {
                set_error("values not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")");
                return SLR_ERR_INVALID_ARG;
            }
        }
    return SLR_OK;
}

// ------------------------------------------------------------------ Section 2.1

slr_status host_dd_order(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts,
                         const int32_t* part, HostSetup& hs) {
    hs.n = n;
    hs.p = nparts;
    // interface: coupled to another part's node; part -1 (a vertex separator) is
    // always interface, and coupling to it keeps a part's node interior
    std::vector<char> iface(n, 0);
    for (int32_t i = 0; i < n; ++i) {
        if (part[i] < 0) { iface[i] = 1; continue; }
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            int32_t j = colind[q];
            if (j != i && part[j] >= 0 && part[j] != part[i]) { iface[i] = 1; break; }
        }
    }
    // counting sort by (is_interface, part), stable in the original index; the
    // separator nodes form a last group after the parts' interfaces
    auto bucket = [&](int32_t i) -> int64_t {
        return part[i] < 0 ? 2 * (int64_t)nparts : (int64_t)iface[i] * nparts + part[i];
    };
    std::vector<int64_t> cnt(2 * (int64_t)nparts + 2, 0);
    for (int32_t i = 0; i < n; ++i) cnt[1 + bucket(i)]++;
    for (size_t t = 1; t < cnt.size(); ++t) cnt[t] += cnt[t - 1];
    hs.int_off.assign(nparts + 1, 0);
    hs.ifc_off.assign(nparts + 1, 0);
    for (int32_t q = 0; q <= nparts; ++q) hs.int_off[q] = (int32_t)cnt[q];
    hs.nI = hs.int_off[nparts];
    for (int32_t q = 0; q <= nparts; ++q) hs.ifc_off[q] = (int32_t)(cnt[nparts + q] - hs.nI);
    hs.s = n - hs.nI;
    hs.perm.assign(n, 0);
    hs.iperm.assign(n, 0);
    std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
    for (int32_t i = 0; i < n; ++i) {
        int32_t d = (int32_t)pos[bucket(i)]++;
        hs.perm[d] = i;
        hs.iperm[i] = d;
    }
    return SLR_OK;
}

slr_status host_split_blocks(const int32_t* rowptr, const int32_t* colind, const double* val,
                             HostSetup& hs) {
    const int32_t n = hs.n, nI = hs.nI, s = hs.s;
    hs.a_rp.assign(n + 1, 0);
    hs.a_ci.resize(rowptr[n]);
    hs.a_v.resize(rowptr[n]);
    std::vector<std::pair<int32_t, double>> row;
    for (int32_t a = 0; a < n; ++a) {
        int32_t i = hs.perm[a];
        row.clear();
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q) row.emplace_back(hs.iperm[colind[q]], val[q]);
        std::sort(row.begin(), row.end(),
                  [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
                      return x.first < y.first;
                  });
        int32_t o = hs.a_rp[a];
        for (auto& e : row) { hs.a_ci[o] = e.first; hs.a_v[o] = e.second; ++o; }
        hs.a_rp[a + 1] = o;
    }
    auto block = [&](int32_t r0, int32_t r1, int32_t c0, int32_t c1, std::vector<int32_t>& rp,
                     std::vector<int32_t>& ci, std::vector<double>& v) {
        rp.assign(r1 - r0 + 1, 0);
        ci.clear();
        v.clear();
        for (int32_t a = r0; a < r1; ++a) {
            for (int32_t q = hs.a_rp[a]; q < hs.a_rp[a + 1]; ++q) {
                int32_t c = hs.a_ci[q];
                if (c >= c0 && c < c1) { ci.push_back(c - c0); v.push_back(hs.a_v[q]); }
            }
            rp[a - r0 + 1] = (int32_t)ci.size();
        }
    };
    block(0, nI, nI, n, hs.e_rp, hs.e_ci, hs.e_v);
    block(nI, n, 0, nI, hs.et_rp, hs.et_ci, hs.et_v);
    block(nI, n, nI, n, hs.c_rp, hs.c_ci, hs.c_v);
    (void)s;
    return SLR_OK;
}

// ------------------------------------------------------------------ Section 5.2: B_i

// Lower-triangular inverse of the W x W matrix D (row-major), into X (row-major):
// X[r][c] = -(sum over q = c .. r-1 of D[r][q] X[q][c]) / D[r][r], X[c][c] = 1 / D[c][c].
// Columns are independent; a block of 16 columns walks the rows with the sums of
// its columns side by side (contiguous in X's rows), each sum over q in ascending
// order, so every entry is the same as computed column by column.
static void tri_inverse(int W, const double* D, double* X) {
    for (int i = 0; i < W * W; ++i) X[i] = 0.0;
    constexpr int CB = 16;
    const int nblk = (W + CB - 1) / CB;
    // threads share a large block (serial inside a parallel region)
#pragma omp parallel for schedule(dynamic, 1) if (W >= 256)
    for (int bk = 0; bk < nblk; ++bk) {
        const int c0 = bk * CB, c1 = std::min(W, c0 + CB);
        double acc[CB];
        for (int r = c0; r < W; ++r) {
            const int ce = std::min(r, c1);          // columns c0 .. ce-1 lie left of the diagonal
            for (int c = c0; c < ce; ++c) acc[c - c0] = 0.0;
            for (int q = c0; q < r; ++q) {           // column c takes the terms q >= c
                const double d = D[r * W + q];
                const double* xq = X + (int64_t)q * W;
                const int qe = std::min(q + 1, ce);
                for (int c = c0; c < qe; ++c) acc[c - c0] += d * xq[c];
            }
            for (int c = c0; c < ce; ++c) X[r * W + c] = -acc[c - c0] / D[r * W + r];
            if (r < c1) X[r * W + r] = 1.0 / D[r * W + r];
        }
    }
}

// Block k of a plane (rows 32 k .. min(32 k + 32, W) - 1) costs sum (W - r) in the
// upper blocks and sum (r + 1) in the lower ones.  Each slice gets at most 8
// blocks; the assignment minimises the larger of the two sums over the slices
// (exhaustively for up to 2^18 assignments, else by dealing blocks from both ends
// round-robin).  Inside a slice, blocks keep ascending order.
void band_assign_blocks(BandBlock& b, int G) {
    const int W = b.w, nb = (W + 31) / 32;
    std::memset(b.nrb, 0, sizeof(b.nrb));
    std::memset(b.rbmap, 0, sizeof(b.rbmap));
    std::vector<int> owner(nb, 0);
    if (G > 1 && nb > 0) {
        std::vector<double> up(nb), lo(nb);
        for (int k = 0; k < nb; ++k)
            for (int r = 32 * k; r < std::min(W, 32 * k + 32); ++r) {
                up[k] += W - r;
                lo[k] += r + 1;
            }
        auto cost = [&](const std::vector<int>& own) {
            double U[4] = {0, 0, 0, 0}, L[4] = {0, 0, 0, 0};
            int cnt[4] = {0, 0, 0, 0};
            for (int k = 0; k < nb; ++k) {
                U[own[k]] += up[k];
                L[own[k]] += lo[k];
                ++cnt[own[k]];
            }
            double c = 0;
            for (int g = 0; g < G; ++g) {
                if (cnt[g] > 8) return 1e300;
                c = std::max(c, std::max(U[g], L[g]));
            }
            return c;
        };
        double total = 1;
        for (int k = 0; k < nb; ++k) total *= G;
        if (total <= double(1 << 18)) {
            std::vector<int> cur(nb, 0);
            double best = 1e301;
            for (long long code = 0; code < (long long)total; ++code) {
                long long x = code;
                for (int k = 0; k < nb; ++k, x /= G) cur[k] = (int)(x % G);
                const double c = cost(cur);
                if (c < best) {
                    best = c;
                    owner = cur;
                }
            }
        } else {
            int g = 0;
            for (int lo_k = 0, hi_k = nb - 1; lo_k <= hi_k; ++lo_k, --hi_k, g = (g + 1) % G) {
                owner[lo_k] = g;
                owner[hi_k] = g;
            }
        }
    }
    for (int k = 0; k < nb; ++k) {
        const int g = owner[k];
        b.rbmap[g][b.nrb[g]++] = (uint8_t)k;
    }
}

std::vector<BandBlock> band_run_order(const std::vector<BandBlock>& band, int mode) {
    std::vector<BandBlock> run(band);
    if (mode <= 1) return run;
    auto work = [](const BandBlock& b) { return (int64_t)b.c * b.w * (b.w + 1); };
    std::stable_sort(run.begin(), run.end(),
                     [&](const BandBlock& a, const BandBlock& b) { return work(a) > work(b); });
    if (mode == 2) return run;
    std::vector<BandBlock> alt;
    alt.reserve(run.size());
    for (size_t lo = 0, hi = run.size(); lo < hi;) {
        alt.push_back(run[lo++]);
        if (lo < hi) alt.push_back(run[--hi]);
    }
    return alt;
}

void host_band_layout(HostSetup& hs, int32_t G) {
    const int32_t p = hs.p;
    hs.band.assign(p, BandBlock());
    hs.band_w.assign(p, 0);
    std::vector<int32_t>& bw = hs.band_w;
    std::map<int32_t, BandBlock> assigned;   // block assignment per plane width
    int64_t off = 0;
    hs.wmax = 0;
    for (int32_t i = 0; i < p; ++i) {
        int32_t r0 = hs.int_off[i], m = hs.int_off[i + 1] - r0, w = 0;
        for (int32_t a = r0; a < r0 + m; ++a)
            for (int32_t q = hs.a_rp[a]; q < hs.a_rp[a + 1]; ++q) {
                int32_t c = hs.a_ci[q];
                if (c >= r0 && c < r0 + m) w = std::max(w, std::abs(a - c));
            }
        bw[i] = w;
        BandBlock& b = hs.band[i];
        b.id = i;
        b.m = m;
        b.row0 = r0;
        b.w = m ? std::max(w, 1) : 0;
        b.c = m ? (m + b.w - 1) / b.w : 0;
        if (m) {
            auto it = assigned.find(b.w);
            if (it == assigned.end()) {
                band_assign_blocks(b, G);
                assigned[b.w] = b;
            } else {
                std::memcpy(b.nrb, it->second.nrb, sizeof(b.nrb));
                std::memcpy(b.rbmap, it->second.rbmap, sizeof(b.rbmap));
            }
        }
        int so = 0, sd = 0;   // segments of the widest slice
        for (int g = 0; g < G; ++g) {
            int a = 0, d = 0;
            for (int rb = 0; rb < b.nrb[g]; ++rb) {
                a += b.w - band_cU0(b, g, rb);
                d += band_cL1(b, g, rb);
            }
            so = std::max(so, a);
            sd = std::max(sd, d);
        }
        b.SU = 32 * so;
        b.SL = 32 * sd;
        b.foff = off;
        off += (int64_t)b.c * G * 2 * (b.SU + b.SL);
        hs.wmax = std::max(hs.wmax, b.w);
    }
    hs.band_G = G;
    hs.bfac_len = off + 64;   // tail slack: bulk copies round up to 16 bytes
}

slr_status host_band_factor(HostSetup& hs, int32_t G) {
    host_band_layout(hs, G);
    const int32_t p = hs.p;
    const std::vector<int32_t>& bw = hs.band_w;
    hs.bfac.assign(hs.bfac_len, 0.0);
    int bad = -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t i = 0; i < p; ++i) {
        const BandBlock& b = hs.band[i];
        const int32_t m = b.m, w = bw[i], W = b.w, r0 = b.row0;
        if (m == 0) continue;
        const int32_t lw = w + 1;
        std::vector<double> Lb((size_t)m * lw, 0.0);  // Lb[l*lw + (k - l + w)] = L[l][k]
        for (int32_t l = 0; l < m; ++l)
            for (int32_t q = hs.a_rp[r0 + l]; q < hs.a_rp[r0 + l + 1]; ++q) {
                int32_t k = hs.a_ci[q] - r0;
                if (k >= 0 && k <= l) Lb[(size_t)l * lw + (k - l + w)] = hs.a_v[q];
            }
        // SPD: B_i = L L^T.  Indefinite (hs.indefinite): B_i = L S L^T with S = diag(sg)
        // the pivot signs (a symmetric factorisation without pivoting), L = Lt |D|^{1/2}.
        std::vector<double> sg((size_t)b.c * W, 1.0);   // plane rows past m keep +1
        const bool indef = hs.indefinite;
        bool ok = true;
        for (int32_t l = 0; l < m && ok; ++l) {
            double* Ll = &Lb[(size_t)l * lw + (w - l)];   // Ll[k] = L[l][k]
            int32_t jlo = std::max(0, l - w);
            for (int32_t j = jlo; j <= l; ++j) {
                const double* Lj = &Lb[(size_t)j * lw + (w - j)];
                int32_t klo = std::max(jlo, j - w);
                double s = Ll[j];
                if (indef)
                    for (int32_t k = klo; k < j; ++k) s -= Ll[k] * sg[k] * Lj[k];
                else
                    for (int32_t k = klo; k < j; ++k) s -= Ll[k] * Lj[k];
                if (j < l) {
                    Ll[j] = s / (sg[j] * Lj[j]);
                } else if (indef) {
                    if (!(std::fabs(s) > 0.0)) { ok = false; break; }
                    sg[l] = s < 0.0 ? -1.0 : 1.0;
                    Ll[l] = std::sqrt(std::fabs(s));
                } else {
                    if (!(s > 0.0)) { ok = false; break; }
                    Ll[l] = std::sqrt(s);
                }
            }
        }
        if (!ok) {
#pragma omp critical
            bad = i;
            continue;
        }
        auto Lat = [&](int32_t l, int32_t k) -> double {   // L[l][k] inside the band, else 0
            if (l < 0 || l >= m || k < 0 || k > l || l - k > w) return 0.0;
            return Lb[(size_t)l * lw + (k - l + w)];
        };
        std::vector<double> D((size_t)W * W), X((size_t)W * W);
        for (int32_t J = 0; J < b.c; ++J) {
            for (int32_t r = 0; r < W; ++r)
                for (int32_t c = 0; c < W; ++c) {
                    int32_t l = J * W + r;
                    D[(size_t)r * W + c] = (l >= m) ? (r == c ? 1.0 : 0.0) : (c <= r ? Lat(l, J * W + c) : 0.0);
                }
            tri_inverse(W, D.data(), X.data());
            double* plane = &hs.bfac[b.foff + (int64_t)J * G * 2 * (b.SU + b.SL)];
            for (int g = 0; g < G; ++g) {
                double* Uf = plane + (int64_t)g * 2 * (b.SU + b.SL);   // O_J      (upper)
                double* Lf = Uf + b.SU;                                 // D_J      (lower)
                double* Lb = Lf + b.SL;                                 // O_J^T    (lower)
                double* Ub = Lb + b.SL;                                 // D_J^T    (upper)
                int64_t su = 0, sl = 0;   // next upper / lower segment
                for (int rb = 0; rb < b.nrb[g]; ++rb) {
                    const int R0 = band_R0(b, g, rb);
                    for (int cc = band_cU0(b, g, rb); cc < W; ++cc, ++su)      // upper: rows r <= cc
                        for (int e = 0; e < 32; ++e) {
                            const int r = R0 + e, l = J * W + r;
                            if (r >= W || r > cc) continue;
                            // forward blocks carry the pivot signs: O_J S_{J-1} and S_J D_J^{-1}
                            Uf[su * 32 + e] = (J > 0 && l < m) ? Lat(l, (J - 1) * W + cc) * sg[(size_t)(J - 1) * W + cc]
                                                               : 0.0;                            // O_J[r][cc]
                            Ub[su * 32 + e] = X[(size_t)cc * W + r];                             // D_J^{-1}[cc][r]
                        }
                    for (int cc = 0; cc < band_cL1(b, g, rb); ++cc, ++sl)      // lower: rows r >= cc
                        for (int e = 0; e < 32; ++e) {
                            const int r = R0 + e, lc = J * W + cc;
                            if (r >= W || r < cc) continue;
                            Lf[sl * 32 + e] = X[(size_t)r * W + cc] * sg[(size_t)J * W + r];     // D_J^{-1}[r][cc]
                            Lb[sl * 32 + e] = (J > 0 && lc < m) ? Lat(lc, (J - 1) * W + r) : 0.0;   // O_J[cc][r]
                        }
                }
            }
        }
    }
    if (bad >= 0) {
        if (hs.indefinite) {
            set_error("B_" + std::to_string(bad) + " has a zero pivot in its symmetric factorisation");
            return SLR_ERR_BREAKDOWN;
        }
        set_error("B_" + std::to_string(bad) + " is not positive definite (Cholesky pivot <= 0)");
        return SLR_ERR_NOT_SPD;
    }
    return SLR_OK;
}

// ------------------------------------------------------------------ Section 3.1: C = L L^T

namespace {

// Nested dissection by breadth-first level structures: a subset is split at the
// middle level of a BFS from a pseudo-peripheral node; both halves are ordered
// first (recursively), the separator last.  Subsets of at most `leaf` nodes,
// and subsets without three levels, become one supernode each.
struct NestedDissection {
    const std::vector<int32_t>& rp;
    const std::vector<int32_t>& ci;
    int32_t leaf;
    std::vector<int32_t> stamp, lev;
    int32_t cur = 0;
    std::vector<int32_t> out_nodes, out_ptr;

    NestedDissection(const std::vector<int32_t>& r, const std::vector<int32_t>& c, int32_t s, int32_t lf)
        : rp(r), ci(c), leaf(lf), stamp(s, 0), lev(s, -1) { out_ptr.push_back(0); }

    void emit(const std::vector<int32_t>& nodes) {
        if (nodes.empty()) return;
        out_nodes.insert(out_nodes.end(), nodes.begin(), nodes.end());
        out_ptr.push_back((int32_t)out_nodes.size());
    }
    int32_t degree(int32_t v) const {
        int32_t d = 0;
        for (int32_t q = rp[v]; q < rp[v + 1]; ++q) d += (stamp[ci[q]] == cur);
        return d;
    }
    // BFS inside the current subset; `order` gets the visit order, lptr level starts.
    void bfs(int32_t root, std::vector<int32_t>& order, std::vector<int32_t>& lptr, int32_t tag) {
        order.clear();
        lptr.clear();
        order.push_back(root);
        lev[root] = tag;
        lptr.push_back(0);
        size_t head = 0;
        while (head < order.size()) {
            size_t end = order.size();
            lptr.push_back((int32_t)end);
            for (; head < end; ++head) {
                int32_t v = order[head];
                for (int32_t q = rp[v]; q < rp[v + 1]; ++q) {
                    int32_t u = ci[q];
                    if (stamp[u] == cur && lev[u] != tag) { lev[u] = tag; order.push_back(u); }
                }
            }
        }
        if (lptr.back() != (int32_t)order.size()) lptr.push_back((int32_t)order.size());
        // remove a trailing empty level marker
        while (lptr.size() >= 2 && lptr[lptr.size() - 1] == lptr[lptr.size() - 2]) lptr.pop_back();
    }
    int32_t tag_counter = 0;

    void run(std::vector<int32_t> nodes) {
        if ((int32_t)nodes.size() <= leaf) { emit(nodes); return; }
        ++cur;
        for (int32_t v : nodes) stamp[v] = cur;
        std::vector<int32_t> order, lptr;
        int32_t tag = ++tag_counter;
        bfs(nodes[0], order, lptr, tag);
        if (order.size() < nodes.size()) {   // several components: order each on its own
            std::vector<std::vector<int32_t>> comps;
            comps.push_back(order);
            for (int32_t v : nodes)
                if (lev[v] != tag) {
                    std::vector<int32_t> o2, l2;
                    bfs(v, o2, l2, tag);
                    comps.push_back(o2);
                }
            for (auto& c : comps) run(c);
            return;
        }
        // pseudo-peripheral root (George & Liu): move to a minimum-degree node of
        // the last level while the eccentricity grows
        int32_t nlev = (int32_t)lptr.size() - 1;
        for (int it = 0; it < 6; ++it) {
            int32_t best = -1, bd = 1 << 30;
            for (int32_t t = lptr[nlev - 1]; t < lptr[nlev]; ++t) {
                int32_t d = degree(order[t]);
                if (d < bd) { bd = d; best = order[t]; }
            }
            std::vector<int32_t> o2, l2;
            int32_t tg = ++tag_counter;
            bfs(best, o2, l2, tg);
            int32_t nl2 = (int32_t)l2.size() - 1;
            if (nl2 > nlev) { order.swap(o2); lptr.swap(l2); nlev = nl2; }
            else break;
        }
        if (nlev < 3) { emit(nodes); return; }
        int32_t half = (int32_t)nodes.size() / 2, mid = 1;
        for (int32_t l = 0; l < nlev; ++l)
            if (lptr[l + 1] > half) { mid = l; break; }
        mid = std::min(std::max(mid, 1), nlev - 2);
        std::vector<int32_t> A(order.begin(), order.begin() + lptr[mid]);
        std::vector<int32_t> S(order.begin() + lptr[mid], order.begin() + lptr[mid + 1]);
        std::vector<int32_t> B(order.begin() + lptr[mid + 1], order.end());
        run(std::move(A));
        run(std::move(B));
        emit(S);
    }
};

}  // namespace

// In-place Cholesky of the lower triangle of the n x n row-major block F (leading
// dimension n); false on a non-positive pivot.  Right-looking in 64-column
// panels: the panel below and the trailing update run in parallel over rows.
static bool chol_blocked(double* F, int32_t n) {
    const int32_t nb = 64;
    for (int32_t k0 = 0; k0 < n; k0 += nb) {
        const int32_t k1 = std::min(n, k0 + nb);
        for (int32_t i = k0; i < k1; ++i) {   // diagonal block (earlier panels applied)
            double* Fi = F + (int64_t)i * n;
            for (int32_t j = k0; j <= i; ++j) {
                const double* Fr = F + (int64_t)j * n;
                double sum = Fi[j];
                for (int32_t k = k0; k < j; ++k) sum -= Fi[k] * Fr[k];
                if (j < i) Fi[j] = sum / Fr[j];
                else if (sum > 0.0) Fi[i] = std::sqrt(sum);
                else return false;
            }
        }
#pragma omp parallel for schedule(static) if ((int64_t)(n - k1) * (k1 - k0) > 8192)
        for (int32_t i = k1; i < n; ++i) {   // panel rows: L[i, k0:k1] = F[i, k0:k1] L_kk^{-T}
            double* Fi = F + (int64_t)i * n;
            for (int32_t j = k0; j < k1; ++j) {
                const double* Fr = F + (int64_t)j * n;
                double sum = Fi[j];
                for (int32_t k = k0; k < j; ++k) sum -= Fi[k] * Fr[k];
                Fi[j] = sum / Fr[j];
            }
        }
#pragma omp parallel for schedule(dynamic, 8) if (n - k1 > 64)
        for (int32_t i = k1; i < n; ++i) {   // trailing lower triangle
            double* Fi = F + (int64_t)i * n;
            for (int32_t j = k1; j <= i; ++j) {
                const double* Fr = F + (int64_t)j * n;
                double dot = 0.0;
                for (int32_t k = k0; k < k1; ++k) dot += Fi[k] * Fr[k];
                Fi[j] -= dot;
            }
        }
    }
    return true;
}

slr_status host_c_factor(HostSetup& hs, int32_t leaf, int32_t task_rows) {
    CFactorHost& cf = hs.cf;
    const int32_t s = hs.s;
    cf = CFactorHost();
    cf.s = s;
    if (s == 0) {
        cf.c0.assign(1, 0);
        cf.r_off.assign(1, 0);
        cf.pan_off.assign(1, 0);
        cf.dinv_off.assign(1, 0);
        cf.seg_ptr.assign(1, 0);
        cf.lev_task_ptr.assign(1, 0);
        cf.lev_ptask_ptr.assign(1, 0);
        cf.lev_sn_ptr.assign(1, 0);
        return SLR_OK;
    }
    // graph of C without its diagonal
    std::vector<int32_t> grp(s + 1, 0), gci;
    for (int32_t a = 0; a < s; ++a) {
        for (int32_t q = hs.c_rp[a]; q < hs.c_rp[a + 1]; ++q)
            if (hs.c_ci[q] != a) gci.push_back(hs.c_ci[q]);
        grp[a + 1] = (int32_t)gci.size();
    }
    NestedDissection nd(grp, gci, s, std::max(leaf, 1));
    {
        std::vector<int32_t> all(s);
        std::iota(all.begin(), all.end(), 0);
        nd.run(std::move(all));
    }
    cf.cperm = nd.out_nodes;
    cf.c0 = nd.out_ptr;
    cf.ns = (int32_t)cf.c0.size() - 1;
    const int32_t ns = cf.ns;
    std::vector<int32_t> ipos(s), snof(s);
    for (int32_t t = 0; t < s; ++t) ipos[cf.cperm[t]] = t;
    for (int32_t J = 0; J < ns; ++J)
        for (int32_t t = cf.c0[J]; t < cf.c0[J + 1]; ++t) snof[t] = J;

    // symbolic: R_J = rows of C below J's columns plus the children's R_K
    cf.parent.assign(ns, -1);
    cf.level.assign(ns, 0);
    cf.r_off.assign(ns + 1, 0);
    std::vector<std::vector<int32_t>> children(ns);
    std::vector<int32_t> mark(s, -1), R;
    for (int32_t J = 0; J < ns; ++J) {
        const int32_t a0 = cf.c0[J], a1 = cf.c0[J + 1];
        R.clear();
        for (int32_t t = a0; t < a1; ++t) {
            int32_t v = cf.cperm[t];
            for (int32_t q = grp[v]; q < grp[v + 1]; ++q) {
                int32_t r = ipos[gci[q]];
                if (r >= a1 && mark[r] != J) { mark[r] = J; R.push_back(r); }
            }
        }
        int32_t lv = 0;
        for (int32_t K : children[J]) {
            lv = std::max(lv, cf.level[K] + 1);
            for (int64_t t = cf.r_off[K]; t < cf.r_off[K + 1]; ++t) {
                int32_t r = cf.rows[t];
                if (r >= a1 && mark[r] != J) { mark[r] = J; R.push_back(r); }
            }
        }
        std::sort(R.begin(), R.end());
        cf.level[J] = lv;
        cf.rows.insert(cf.rows.end(), R.begin(), R.end());
        cf.r_off[J + 1] = (int64_t)cf.rows.size();
        if (!R.empty()) {
            cf.parent[J] = snof[R[0]];
            children[cf.parent[J]].push_back(J);
        }
    }
    // numeric: right-looking supernodal Cholesky on dense panels
    // F_J: (n_J + |R_J|) x n_J row-major; the first n_J rows are the diagonal block
    std::vector<int64_t> fo(ns + 1, 0);
    for (int32_t J = 0; J < ns; ++J) {
        int64_t nJ = cf.c0[J + 1] - cf.c0[J], nr = cf.r_off[J + 1] - cf.r_off[J];
        fo[J + 1] = fo[J] + (nJ + nr) * nJ;
    }
    std::vector<double> F(fo[ns], 0.0);
    auto rowpos = [&](int32_t T, int32_t r) -> int64_t {   // row of position r inside F_T
        if (r < cf.c0[T + 1]) return r - cf.c0[T];
        const int32_t* b = cf.rows.data() + cf.r_off[T];
        const int32_t* e = cf.rows.data() + cf.r_off[T + 1];
        const int32_t* f = std::lower_bound(b, e, r);
        return (cf.c0[T + 1] - cf.c0[T]) + (f - b);
    };
    for (int32_t J = 0; J < ns; ++J) {
        const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
        for (int32_t t = a0; t < a0 + nJ; ++t) {
            int32_t v = cf.cperm[t];
            for (int32_t q = hs.c_rp[v]; q < hs.c_rp[v + 1]; ++q) {
                int32_t r = ipos[hs.c_ci[q]];
                if (r < t) continue;
                F[fo[J] + rowpos(J, r) * nJ + (t - a0)] += hs.c_v[q];
            }
        }
    }
    int bad = -1;
    for (int32_t J = 0; J < ns && bad < 0; ++J) {
        const int32_t a0 = cf.c0[J], nJ = cf.c0[J + 1] - a0;
        const int64_t nr = cf.r_off[J + 1] - cf.r_off[J];
        double* Fj = F.data() + fo[J];
        if (nJ >= 128) {   // large diagonal block: blocked, with parallel panels and updates
            if (!chol_blocked(Fj, nJ)) bad = J;
        }
        for (int32_t i = 0; i < nJ && bad < 0 && nJ < 128; ++i) {
            double* Fi = Fj + (int64_t)i * nJ;
            for (int32_t j = 0; j <= i; ++j) {
                const double* Fr = Fj + (int64_t)j * nJ;
                double sum = Fi[j];
                for (int32_t k = 0; k < j; ++k) sum -= Fi[k] * Fr[k];
                if (j < i) Fi[j] = sum / Fr[j];
                else if (sum > 0.0) Fi[i] = std::sqrt(sum);
                else { bad = J; break; }
            }
        }
        if (bad >= 0) break;
        // panel rows L[R_J, J] = F[R_J, J] L_JJ^{-T}, four rows per pass: four independent
        // chains, each row's sum in the same order as alone
#pragma omp parallel for schedule(static) if (nr * nJ > 4096)
        for (int64_t p4 = 0; p4 < (nr + 3) / 4; ++p4) {
            const int64_t pr = 4 * p4;
            if (pr + 4 <= nr) {
                double* F0 = Fj + (nJ + pr) * nJ;
                double *F1 = F0 + nJ, *F2 = F1 + nJ, *F3 = F2 + nJ;
                for (int32_t j = 0; j < nJ; ++j) {
                    const double* Fr = Fj + (int64_t)j * nJ;
                    double s0 = F0[j], s1 = F1[j], s2 = F2[j], s3 = F3[j];
                    for (int32_t k = 0; k < j; ++k) {
                        const double r = Fr[k];
                        s0 -= F0[k] * r;
                        s1 -= F1[k] * r;
                        s2 -= F2[k] * r;
                        s3 -= F3[k] * r;
                    }
                    F0[j] = s0 / Fr[j];
                    F1[j] = s1 / Fr[j];
                    F2[j] = s2 / Fr[j];
                    F3[j] = s3 / Fr[j];
                }
            } else {
                for (int64_t q = pr; q < nr; ++q) {
                    double* Fp = Fj + (nJ + q) * nJ;
                    for (int32_t j = 0; j < nJ; ++j) {
                        const double* Fr = Fj + (int64_t)j * nJ;
                        double sum = Fp[j];
                        for (int32_t k = 0; k < j; ++k) sum -= Fp[k] * Fr[k];
                        Fp[j] = sum / Fr[j];
                    }
                }
            }
        }
        // update the ancestors: F_T[R_J[a], R_J[b]] -= L[R_J[a], J] . L[R_J[b], J]
        const int32_t* RJ = cf.rows.data() + cf.r_off[J];
        int64_t b0 = 0;
        while (b0 < nr) {
            const int32_t T = snof[RJ[b0]];
            int64_t b1 = b0;
            while (b1 < nr && RJ[b1] < cf.c0[T + 1]) ++b1;
            const int32_t nT = cf.c0[T + 1] - cf.c0[T];
            double* FT = F.data() + fo[T];
            // row a of F_T (position R_J[a]) -= L[R_J[a], J] . L[R_J[b], J] for b0 <= b <= a, b < b1;
            // every dot runs over k in ascending order whatever the tiling
            auto dots = [&](int64_t a, int64_t bs, int64_t be) {
                const double* La = Fj + (nJ + a) * nJ;
                const int64_t fb = rowpos(T, RJ[a]) * nT - cf.c0[T];   // F_T[row of R_J[a], col] at fb + col
                int64_t b = bs;
                for (; b + 4 <= be; b += 4) {   // four dots per pass over La
                    const double* L0 = Fj + (nJ + b) * nJ;
                    const double *L1 = L0 + nJ, *L2 = L1 + nJ, *L3 = L2 + nJ;
                    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
                    for (int32_t k = 0; k < nJ; ++k) {
                        const double x = La[k];
                        d0 += x * L0[k];
                        d1 += x * L1[k];
                        d2 += x * L2[k];
                        d3 += x * L3[k];
                    }
                    FT[fb + RJ[b]] -= d0;
                    FT[fb + RJ[b + 1]] -= d1;
                    FT[fb + RJ[b + 2]] -= d2;
                    FT[fb + RJ[b + 3]] -= d3;
                }
                for (; b < be; ++b) {
                    const double* Lbr = Fj + (nJ + b) * nJ;
                    double dot = 0.0;
                    for (int32_t k = 0; k < nJ; ++k) dot += La[k] * Lbr[k];
                    FT[fb + RJ[b]] -= dot;
                }
            };
            // four rows a at a time: 4 x 4 tiles of dots over the b they all take (each
            // row of the panel is then read once per four dots), the rest row by row
            const int64_t ngrp = (nr - b0 + 3) / 4;
#pragma omp parallel for schedule(dynamic, 4) if ((nr - b0) * (b1 - b0) * nJ > 100000)
            for (int64_t gi = 0; gi < ngrp; ++gi) {
                const int64_t a0 = b0 + 4 * gi, a1 = std::min(nr, a0 + 4);
                int64_t bt = b0;   // tiles cover b0 .. bt-1 for every row of the group
                if (a1 - a0 == 4) {
                    const int64_t btile = std::min(a0 + 1, b1);   // every row of the group takes b < btile
                    const double* A0 = Fj + (nJ + a0) * nJ;
                    const double *A1 = A0 + nJ, *A2 = A1 + nJ, *A3 = A2 + nJ;
                    int64_t fa[4];
                    for (int u = 0; u < 4; ++u) fa[u] = rowpos(T, RJ[a0 + u]) * nT - cf.c0[T];
                    for (; bt + 4 <= btile; bt += 4) {
                        const double* B0 = Fj + (nJ + bt) * nJ;
                        const double *B1 = B0 + nJ, *B2 = B1 + nJ, *B3 = B2 + nJ;
                        double d[4][4] = {};
                        for (int32_t k = 0; k < nJ; ++k) {
                            const double x0 = A0[k], x1 = A1[k], x2 = A2[k], x3 = A3[k];
                            const double y0 = B0[k], y1 = B1[k], y2 = B2[k], y3 = B3[k];
                            d[0][0] += x0 * y0; d[0][1] += x0 * y1; d[0][2] += x0 * y2; d[0][3] += x0 * y3;
                            d[1][0] += x1 * y0; d[1][1] += x1 * y1; d[1][2] += x1 * y2; d[1][3] += x1 * y3;
                            d[2][0] += x2 * y0; d[2][1] += x2 * y1; d[2][2] += x2 * y2; d[2][3] += x2 * y3;
                            d[3][0] += x3 * y0; d[3][1] += x3 * y1; d[3][2] += x3 * y2; d[3][3] += x3 * y3;
                        }
                        for (int u = 0; u < 4; ++u)
                            for (int v = 0; v < 4; ++v) FT[fa[u] + RJ[bt + v]] -= d[u][v];
                    }
                }
                for (int64_t a = a0; a < a1; ++a) dots(a, bt, std::min(a + 1, b1));
            }
            b0 = b1;
        }
    }
    if (bad >= 0) {
        set_error("C is not positive definite (Cholesky pivot <= 0 in supernode " + std::to_string(bad) + ")");
        return SLR_ERR_NOT_SPD;
    }
    // inverted diagonal blocks (packed lower, column-major) and row-major panels M_J
    cf.dinv_off.assign(ns + 1, 0);
    cf.pan_off.assign(ns + 1, 0);
    for (int32_t J = 0; J < ns; ++J) {
        int64_t nJ = cf.c0[J + 1] - cf.c0[J], nr = cf.r_off[J + 1] - cf.r_off[J];
        cf.dinv_off[J + 1] = cf.dinv_off[J] + nJ * (nJ + 1) / 2;
        cf.pan_off[J + 1] = cf.pan_off[J] + nr * nJ;
    }
    cf.dinv.assign(cf.dinv_off[ns], 0.0);
    cf.panel.assign(cf.pan_off[ns], 0.0);
    // small supernodes in parallel, large ones (nJ >= 256) one at a time with
    // parallel loops inside (tri_inverse's columns, M_J's rows)
    auto inv_and_m = [&](int32_t J) {
        const int32_t nJ = cf.c0[J + 1] - cf.c0[J];
        const int64_t nr = cf.r_off[J + 1] - cf.r_off[J];
        const double* Fj = F.data() + fo[J];
        std::vector<double> X((size_t)nJ * nJ);
        tri_inverse(nJ, Fj, X.data());   // Fj's upper part is zero: it is never written
        double* Dv = cf.dinv.data() + cf.dinv_off[J];
        for (int32_t j = 0; j < nJ; ++j) {
            int64_t cs = (int64_t)j * nJ - (int64_t)j * (j - 1) / 2;
            for (int32_t i = j; i < nJ; ++i) Dv[cs + (i - j)] = X[(size_t)i * nJ + j];
        }
        // M_J = L[R_J, J] L_JJ^{-1}: the off-diagonal block of the unit block factor
        // Lhat = L D^{-1}, D = diag(L_JJ), so C = Lhat D D^T Lhat^T (a block LDL^T form)
        const double* Pj = Fj + (int64_t)nJ * nJ;
        double* Mj = cf.panel.data() + cf.pan_off[J];
        // eight panel rows per pass over each row of X (X is read once per eight rows
        // instead of once per row); every M_J entry still sums k in ascending order
        constexpr int64_t RB = 8;
#pragma omp parallel for schedule(static) if (nJ >= 256 && nr >= 16)
        for (int64_t pb = 0; pb < (nr + RB - 1) / RB; ++pb) {
            const int64_t p0 = pb * RB, p1 = std::min(nr, p0 + RB);
            for (int32_t k = 0; k < nJ; ++k) {
                const double* Xk = X.data() + (size_t)k * nJ;
                for (int64_t pr = p0; pr < p1; ++pr) {
                    const double a = Pj[pr * nJ + k];
                    double* Mp = Mj + pr * nJ;
                    for (int32_t j = 0; j <= k; ++j) Mp[j] += a * Xk[j];
                }
            }
        }
    };
#pragma omp parallel for schedule(dynamic, 1)
    for (int32_t J = 0; J < ns; ++J)
        if (cf.c0[J + 1] - cf.c0[J] < 256) inv_and_m(J);
    for (int32_t J = 0; J < ns; ++J)
        if (cf.c0[J + 1] - cf.c0[J] >= 256) inv_and_m(J);
    // forward gather lists: row i of L left of its diagonal block is the union of
    // the panel rows R_K[p] = i of its descendants K
    cf.seg_ptr.assign(s + 1, 0);
    for (int32_t J = 0; J < ns; ++J)
        for (int64_t t = cf.r_off[J]; t < cf.r_off[J + 1]; ++t) cf.seg_ptr[cf.rows[t] + 1]++;
    for (int32_t i = 0; i < s; ++i) cf.seg_ptr[i + 1] += cf.seg_ptr[i];
    cf.seg_row.assign(cf.seg_ptr[s], 0);
    {
        std::vector<int64_t> fill(cf.seg_ptr.begin(), cf.seg_ptr.end() - 1);
        for (int32_t J = 0; J < ns; ++J)
            for (int64_t t = cf.r_off[J]; t < cf.r_off[J + 1]; ++t) cf.seg_row[fill[cf.rows[t]]++] = (int32_t)t;
    }
    // level schedule: column blocks and panel-row blocks of at most task_rows
    cf.nlev = 0;
    for (int32_t J = 0; J < ns; ++J) cf.nlev = std::max(cf.nlev, cf.level[J] + 1);
    std::vector<std::vector<int32_t>> bylev(cf.nlev);
    for (int32_t J = 0; J < ns; ++J) bylev[cf.level[J]].push_back(J);
    cf.lev_task_ptr.assign(cf.nlev + 1, 0);
    cf.lev_ptask_ptr.assign(cf.nlev + 1, 0);
    cf.tasks.clear();
    cf.ptasks.clear();
    auto add = [&](std::vector<int32_t>& v, int32_t J, int32_t n) {
        for (int32_t f = 0; f < n; f += task_rows) {
            v.push_back(J);
            v.push_back(f);
            v.push_back(std::min(task_rows, n - f));
            v.push_back(0);
        }
    };
    for (int32_t l = 0; l < cf.nlev; ++l) {
        for (int32_t J : bylev[l]) {
            add(cf.tasks, J, cf.c0[J + 1] - cf.c0[J]);
            add(cf.ptasks, J, (int32_t)(cf.r_off[J + 1] - cf.r_off[J]));
        }
        cf.lev_task_ptr[l + 1] = (int32_t)(cf.tasks.size() / 4);
        cf.lev_ptask_ptr[l + 1] = (int32_t)(cf.ptasks.size() / 4);
    }
    cf.lev_sn_ptr.assign(cf.nlev + 1, 0);
    cf.lev_sn.clear();
    // One CTA per supernode pays off only when a level has at least a wave of
    // supernodes and each one's panel is small; otherwise the split kernels
    // spread a supernode's rows over many CTAs.
    cf.lev_small.assign(cf.nlev, 1);
    for (int32_t l = 0; l < cf.nlev; ++l) {
        if ((int32_t)bylev[l].size() < kSmallMinCount) cf.lev_small[l] = 0;
        for (int32_t J : bylev[l]) {
            cf.lev_sn.push_back(J);
            const int64_t nJ = cf.c0[J + 1] - cf.c0[J], nr = cf.r_off[J + 1] - cf.r_off[J];
            if (nJ > kSmallN || nr > kSmallR || nJ * nr > kSmallPanel) cf.lev_small[l] = 0;
        }
        cf.lev_sn_ptr[l + 1] = (int32_t)cf.lev_sn.size();
    }
    return SLR_OK;
}

// ------------------------------------------------------------------ top zone (partitioned inverse)

// Entries of L_TT^{-1} (block columns over each supernode's path to the root)
// and the multiply-adds that build it, for the zone of levels >= L.
static void top_zone_cost(const CFactorHost& cf, int32_t L, double* entries, double* fmas) {
    double e = 0.0, f = 0.0;
    for (int32_t J = 0; J < cf.ns; ++J) {
        if (cf.level[J] < L) continue;
        const double nJ = cf.c0[J + 1] - cf.c0[J];
        double below = nJ;
        e += nJ * (nJ + 1) / 2;
        f += nJ * nJ * nJ / 2;
        for (int32_t A = cf.parent[J]; A >= 0; A = cf.parent[A]) {
            const double nA = cf.c0[A + 1] - cf.c0[A];
            e += nA * nJ;
            f += nA * below * nJ + nA * nA / 2 * nJ;
            below += nA;
        }
    }
    *entries = e;
    *fmas = f;
}

int32_t host_c_top_choose(const CFactorHost& cf) {
    const double fac = (double)cf.panel.size() + (double)cf.dinv.size();
    int32_t best = cf.nlev;
    for (int32_t L = cf.nlev - 1; L >= 0; --L) {
        double e = 0.0, f = 0.0;
        top_zone_cost(cf, L, &e, &f);
        if (e > kTopEntries * fac || f > kTopFmas) break;
        best = L;
    }
    return cf.nlev - best >= 2 ? best : cf.nlev;   // a zone of one level saves no step
}

void host_c_top(CFactorHost& cf, int32_t top_lev) {
    cf.top_lev = cf.nlev;
    cf.nT = 0;
    cf.tpos.clear(); cf.tseg_ptr.assign(1, 0); cf.tseg_row.clear();
    cf.tsk_off.assign(1, 0); cf.tsk_lo.clear(); cf.tsk.clear();
    cf.tf_rb.clear(); cf.tf_tasks.clear();
    cf.tb_off.assign(cf.ns + 1, 0); cf.tb.clear(); cf.tp_off.assign(cf.ns + 1, 0); cf.tp_pos.clear();
    cf.tb_cb.clear(); cf.tb_cb_part.clear(); cf.tb_tasks.clear();
    cf.tf_parts = cf.tb_parts = 0;
    if (top_lev >= cf.nlev) return;
    const int32_t ns = cf.ns, s = cf.s;
    std::vector<uint8_t> inT(ns, 0);
    std::vector<int32_t> Tl;   // zone supernodes, ascending (children before parents)
    for (int32_t J = 0; J < ns; ++J)
        if (cf.level[J] >= top_lev) { inT[J] = 1; Tl.push_back(J); }
    std::vector<int32_t> snof(s), loc(s, -1);
    for (int32_t J = 0; J < ns; ++J)
        for (int32_t t = cf.c0[J]; t < cf.c0[J + 1]; ++t) snof[t] = J;
    std::vector<int32_t> tpos;
    for (int32_t t = 0; t < s; ++t)
        if (inT[snof[t]]) { loc[t] = (int32_t)tpos.size(); tpos.push_back(t); }
    const int32_t nT = (int32_t)tpos.size();
    // lo[A] = first local index of the zone within A's subtree; the subtree must
    // fill lo[A] .. (A's last local index) exactly
    std::vector<int32_t> lo(ns, 0);
    std::vector<int64_t> sz(ns, 0);
    for (int32_t J : Tl) { lo[J] = loc[cf.c0[J]]; sz[J] = cf.c0[J + 1] - cf.c0[J]; }
    for (int32_t J : Tl) {
        const int32_t A = cf.parent[J];
        if (A < 0) continue;
        if (!inT[A]) return;   // cannot happen: a parent's level is above its child's
        lo[A] = std::min(lo[A], lo[J]);
        sz[A] += sz[J];
    }
    for (int32_t A : Tl)
        if ((int64_t)loc[cf.c0[A + 1] - 1] - lo[A] + 1 != sz[A]) return;   // not contiguous: no zone
    // block columns X_J = L_TT^{-1}[path_J, J] with the unit block factor Lhat = L D^{-1}:
    // Z = Lhat_TT^{-1}[path_J, J] (Z_J = I, Z_A = - sum_K M_K[rows in A] Z_K over the path
    // below A), then X_A = L_AA^{-1} Z_A
    std::vector<int64_t> plen(ns, 0);
    for (int32_t J : Tl) {
        for (int32_t A = J; A >= 0; A = cf.parent[A]) plen[J] += cf.c0[A + 1] - cf.c0[A];
        const int64_t nJ = cf.c0[J + 1] - cf.c0[J];
        cf.tb_off[J + 1] = nJ * plen[J];
        cf.tp_off[J + 1] = plen[J];
    }
    for (int32_t J = 0; J < ns; ++J) {
        cf.tb_off[J + 1] += cf.tb_off[J];
        cf.tp_off[J + 1] += cf.tp_off[J];
    }
    cf.tb.assign(cf.tb_off[ns], 0.0);
    cf.tp_pos.assign(cf.tp_off[ns], 0);
#pragma omp parallel for schedule(dynamic, 1)
    for (size_t idx = 0; idx < Tl.size(); ++idx) {
        const int32_t J = Tl[idx];   // children first: the long paths start early
        const int32_t nJ = cf.c0[J + 1] - cf.c0[J];
        std::vector<int32_t> path;
        std::vector<int64_t> po;
        int64_t rows = 0;
        for (int32_t A = J; A >= 0; A = cf.parent[A]) {
            path.push_back(A);
            po.push_back(rows);
            rows += cf.c0[A + 1] - cf.c0[A];
        }
        std::vector<double> Z((size_t)rows * nJ, 0.0);
        for (int32_t q = 0; q < nJ; ++q) Z[(size_t)q * nJ + q] = 1.0;
        for (size_t i = 1; i < path.size(); ++i) {
            const int32_t A = path[i], a0 = cf.c0[A], nA = cf.c0[A + 1] - a0;
            double* ZA = Z.data() + po[i] * nJ;
            for (size_t k = 0; k < i; ++k) {
                const int32_t K = path[k], nK = cf.c0[K + 1] - cf.c0[K];
                const int32_t* Rk = cf.rows.data() + cf.r_off[K];
                const int64_t nrK = cf.r_off[K + 1] - cf.r_off[K];
                const int64_t pb = std::lower_bound(Rk, Rk + nrK, a0) - Rk;
                const int64_t pe = std::lower_bound(Rk, Rk + nrK, a0 + nA) - Rk;
                const double* MK = cf.panel.data() + cf.pan_off[K];
                const double* ZK = Z.data() + po[k] * nJ;
                for (int64_t p = pb; p < pe; ++p) {
                    double* zr = ZA + (int64_t)(Rk[p] - a0) * nJ;
                    const double* mrow = MK + p * nK;
                    int32_t q = 0;
                    for (; q + 3 < nK; q += 4) {   // four rows of Z_K per pass over zr
                        const double m0 = mrow[q], m1 = mrow[q + 1], m2 = mrow[q + 2], m3 = mrow[q + 3];
                        const double* z0 = ZK + (int64_t)q * nJ;
                        const double *z1 = z0 + nJ, *z2 = z1 + nJ, *z3 = z2 + nJ;
                        for (int32_t c = 0; c < nJ; ++c) zr[c] -= (m0 * z0[c] + m1 * z1[c]) + (m2 * z2[c] + m3 * z3[c]);
                    }
                    for (; q < nK; ++q) {
                        const double m = mrow[q];
                        const double* zk = ZK + (int64_t)q * nJ;
                        for (int32_t c = 0; c < nJ; ++c) zr[c] -= m * zk[c];
                    }
                }
            }
        }
        double* X = cf.tb.data() + cf.tb_off[J];
        int32_t* pp = cf.tp_pos.data() + cf.tp_off[J];
        for (size_t i = 0; i < path.size(); ++i) {
            const int32_t A = path[i], nA = cf.c0[A + 1] - cf.c0[A];
            const double* Dv = cf.dinv.data() + cf.dinv_off[A];
            auto dv = [&](int32_t a, int32_t b) { return Dv[(int64_t)b * nA - (int64_t)b * (b - 1) / 2 + (a - b)]; };
            for (int32_t a = 0; a < nA; ++a) {
                double* xr = X + (po[i] + a) * nJ;
                const double* zb = Z.data() + po[i] * nJ;
                int32_t b = 0;
                for (; b + 3 <= a; b += 4) {
                    const double d0 = dv(a, b), d1 = dv(a, b + 1), d2 = dv(a, b + 2), d3 = dv(a, b + 3);
                    const double* z0 = zb + (int64_t)b * nJ;
                    const double *z1 = z0 + nJ, *z2 = z1 + nJ, *z3 = z2 + nJ;
                    for (int32_t c = 0; c < nJ; ++c) xr[c] += (d0 * z0[c] + d1 * z1[c]) + (d2 * z2[c] + d3 * z3[c]);
                }
                for (; b <= a; ++b) {
                    const double d = dv(a, b);
                    const double* z = zb + (int64_t)b * nJ;
                    for (int32_t c = 0; c < nJ; ++c) xr[c] += d * z[c];
                }
                pp[po[i] + a] = cf.c0[A] + a;
            }
        }
    }
    // forward row skyline of the same entries
    cf.tsk_lo.assign(nT, 0);
    cf.tsk_off.assign(nT + 1, 0);
    for (int32_t la = 0; la < nT; ++la) {
        cf.tsk_lo[la] = lo[snof[tpos[la]]];
        cf.tsk_off[la + 1] = cf.tsk_off[la] + (la - cf.tsk_lo[la] + 1);
    }
    cf.tsk.assign(cf.tsk_off[nT], 0.0);
#pragma omp parallel for schedule(dynamic, 1)
    for (size_t idx = 0; idx < Tl.size(); ++idx) {
        const int32_t J = Tl[idx], nJ = cf.c0[J + 1] - cf.c0[J];
        const double* X = cf.tb.data() + cf.tb_off[J];
        const int32_t* pp = cf.tp_pos.data() + cf.tp_off[J];
        const int64_t rows = cf.tp_off[J + 1] - cf.tp_off[J];
        for (int64_t r = 0; r < rows; ++r) {
            const int32_t la = loc[pp[r]];
            for (int32_t q = 0; q < nJ; ++q) {
                const int32_t lc = loc[cf.c0[J] + q];
                if (lc <= la) cf.tsk[cf.tsk_off[la] + (lc - cf.tsk_lo[la])] = X[r * nJ + q];
            }
        }
    }
    // gather lists of the zone's rows: contributions of supernodes outside the zone
    std::vector<int32_t> prow_sn(cf.rows.size());
    for (int32_t K = 0; K < ns; ++K)
        for (int64_t t = cf.r_off[K]; t < cf.r_off[K + 1]; ++t) prow_sn[t] = K;
    cf.tseg_ptr.assign(nT + 1, 0);
    for (int32_t la = 0; la < nT; ++la) {
        const int32_t pos = tpos[la];
        for (int64_t e = cf.seg_ptr[pos]; e < cf.seg_ptr[pos + 1]; ++e)
            if (!inT[prow_sn[cf.seg_row[e]]]) cf.tseg_row.push_back(cf.seg_row[e]);
        cf.tseg_ptr[la + 1] = (int64_t)cf.tseg_row.size();
    }
    // forward tasks: 32-row blocks within a supernode, their columns lo .. last row in chunks
    for (int32_t A : Tl) {
        const int32_t l0 = loc[cf.c0[A]], l1 = loc[cf.c0[A + 1] - 1] + 1;
        for (int32_t r0 = l0; r0 < l1; r0 += 32) {
            const int32_t cnt = std::min(32, l1 - r0), clo = lo[A], chi = r0 + cnt;
            const int32_t nch = (chi - clo + kTopCW - 1) / kTopCW;
            const int32_t rb = (int32_t)(cf.tf_rb.size() / 4);
            cf.tf_rb.insert(cf.tf_rb.end(), {r0, cnt, nch, cf.tf_parts});
            for (int32_t k = 0; k < nch; ++k)
                cf.tf_tasks.insert(cf.tf_tasks.end(), {rb, clo + k * kTopCW, std::min(chi, clo + (k + 1) * kTopCW), k});
            cf.tf_parts += 32 * nch;
        }
    }
    // backward tasks: 32-column blocks of J, their path rows (from the block's first
    // column down: the rows above it in J's diagonal block are zero) in chunks
    for (int32_t J : Tl) {
        const int32_t nJ = cf.c0[J + 1] - cf.c0[J];
        const int64_t rows = cf.tp_off[J + 1] - cf.tp_off[J];
        for (int32_t c0 = 0; c0 < nJ; c0 += 32) {
            const int32_t cnt = std::min(32, nJ - c0);
            const int32_t nch = (int32_t)((rows - c0 + kTopRCH - 1) / kTopRCH);
            const int32_t cb = (int32_t)(cf.tb_cb.size() / 4);
            cf.tb_cb.insert(cf.tb_cb.end(), {J, c0, cnt, nch});
            cf.tb_cb_part.push_back(cf.tb_parts);
            for (int32_t k = 0; k < nch; ++k)
                cf.tb_tasks.insert(cf.tb_tasks.end(),
                                   {cb, (int32_t)(c0 + (int64_t)k * kTopRCH),
                                    (int32_t)std::min<int64_t>(rows, c0 + (int64_t)(k + 1) * kTopRCH), k});
            cf.tb_parts += 32 * nch;
        }
    }
    cf.tpos = std::move(tpos);
    cf.nT = nT;
    cf.top_lev = top_lev;
}

// ------------------------------------------------------------------ Section 5.1: T = Y diag(lam) Y^T

// Implicit QL iteration with Wilkinson shifts on the symmetric tridiagonal T
// (Bowdler, Martin, Reinsch & Wilkinson, 1968): each sweep chases a bulge up from
// the bottom of the unreduced block with Givens rotations, which are accumulated
// into the eigenvector rows; a sub-diagonal entry below eps (|d_i| + |d_{i+1}|)
// splits the matrix.  O(m^2) work per eigenvalue with its vector.
void host_tridiag_eig(int32_t m, const double* alpha, const double* beta, double* lam, double* Y) {
    if (m <= 0) return;
    std::vector<double> d(alpha, alpha + m), e(m, 0.0);
    for (int32_t i = 0; i + 1 < m; ++i) e[i] = beta[i];   // e[i] couples d[i] and d[i+1]
    std::vector<double> Z((size_t)m * m, 0.0);             // row i: eigenvector of d[i]
    for (int32_t i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
    const double eps = std::numeric_limits<double>::epsilon();
    for (int32_t l = 0; l < m; ++l) {
        for (int iter = 0; iter < 60; ++iter) {
            int32_t q = l;   // end of the unreduced block that starts at l
            while (q + 1 < m && std::fabs(e[q]) > eps * (std::fabs(d[q]) + std::fabs(d[q + 1]))) ++q;
            if (q == l) break;
            // shift: the eigenvalue of the leading 2 x 2 block nearer d[l]
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = std::hypot(g, 1.0);
            g = d[q] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
            double sn = 1.0, cs = 1.0, p = 0.0;
            int32_t i = q - 1;
            bool split = false;
            for (; i >= l; --i) {
                const double f = sn * e[i], bb = cs * e[i];
                r = std::hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {   // the rotation vanished: the block splits at i + 1
                    d[i + 1] -= p;
                    e[q] = 0.0;
                    split = true;
                    break;
                }
                sn = f / r;
                cs = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * sn + 2.0 * cs * bb;
                p = sn * r;
                d[i + 1] = g + p;
                g = cs * r - bb;
                double* zi = Z.data() + (size_t)i * m;
                double* zj = zi + m;
                for (int32_t k = 0; k < m; ++k) {
                    const double zk = zj[k];
                    zj[k] = sn * zi[k] + cs * zk;
                    zi[k] = cs * zi[k] - sn * zk;
                }
            }
            if (split) continue;
            d[l] -= p;
            e[l] = g;
            e[q] = 0.0;
        }
    }
    std::vector<int32_t> idx(m);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return d[a] > d[b]; });
    for (int32_t j = 0; j < m; ++j) {
        lam[j] = d[idx[j]];
        std::memcpy(Y + (size_t)j * m, Z.data() + (size_t)idx[j] * m, sizeof(double) * m);
    }
}

}  // namespace slr

// ------------------------------------------------------------------ host-only ABI entries

extern "C" {

void slr_default_opts(slr_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->k = 16;
    o->lanczos_steps = 0;
    o->theta_mode = SLR_THETA_LAMBDA_K1;
    o->precision = SLR_PREC_FP64;
    o->nrhs_max = 1;
    o->flexible_cg = 0;
    o->seed = 1;
    o->c_leaf = 64;
}

const char* slr_status_str(slr_status s) {
    switch (s) {
        case SLR_OK: return "SLR_OK";
        case SLR_ERR_INVALID_ARG: return "SLR_ERR_INVALID_ARG";
        case SLR_ERR_NOT_SPD: return "SLR_ERR_NOT_SPD";
        case SLR_ERR_OOM: return "SLR_ERR_OOM";
        case SLR_ERR_CUDA: return "SLR_ERR_CUDA";
        case SLR_ERR_NOT_CONVERGED: return "SLR_ERR_NOT_CONVERGED";
        case SLR_ERR_BREAKDOWN: return "SLR_ERR_BREAKDOWN";
        case SLR_ERR_TIMEOUT: return "SLR_ERR_TIMEOUT";
        case SLR_ERR_UNSUPPORTED: return "SLR_ERR_UNSUPPORTED";
    }
    return "SLR_ERR_UNKNOWN";
}

const char* slr_last_error_message(void) { return slr::g_last_error.c_str(); }

slr_status slr_dd_order(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t nparts,
                        const int32_t* part, int32_t* perm_out, int32_t* int_off, int32_t* ifc_off,
                        int32_t* s_out) {
    if (n < 0 || nparts < 1 || (n > 0 && (!rowptr || !part || (rowptr[n] > 0 && !colind)))) {
        slr::set_error("invalid arguments");
        return SLR_ERR_INVALID_ARG;
    }
    for (int32_t i = 0; i < n; ++i)
        if (part[i] < -1 || part[i] >= nparts) { slr::set_error("part out of range"); return SLR_ERR_INVALID_ARG; }
    for (int32_t i = 0; i < n; ++i)
        for (int32_t q = rowptr[i]; q < rowptr[i + 1]; ++q)
            if (colind[q] < 0 || colind[q] >= n) { slr::set_error("column out of range"); return SLR_ERR_INVALID_ARG; }
    slr::HostSetup hs;
    slr_status st = slr::host_dd_order(n, rowptr, colind, nparts, part, hs);
    if (st != SLR_OK) return st;
    if (perm_out) std::memcpy(perm_out, hs.perm.data(), sizeof(int32_t) * n);
    if (int_off) std::memcpy(int_off, hs.int_off.data(), sizeof(int32_t) * (nparts + 1));
    if (ifc_off) std::memcpy(ifc_off, hs.ifc_off.data(), sizeof(int32_t) * (nparts + 1));
    if (s_out) *s_out = hs.s;
    return SLR_OK;
}

}  // extern "C"
