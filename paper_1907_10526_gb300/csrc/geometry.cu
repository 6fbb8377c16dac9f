// geometry.cu -- validation and device tables of a fan-beam geometry (Sec. II.A, Eq. 17).
//
// Everything here runs once per geometry, on the host, in FP64.  The per-(view, cell)
// walk of the forward projector is converted to 32.32 fixed point and every walk is
// checked, with the same integer arithmetic the kernel uses, to stay inside the
// zero-padded image copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cnsf.h"
#include "cnsf_internal.cuh"
#include "cnsf_runtime.h"

namespace cnsf {

static inline long long ceil_fx(long long a)   // ceil(a / 2^32)
{
    long long hi = a >> 32;
    return hi + (((unsigned long long)a & 0xffffffffull) != 0ull ? 1 : 0);
}

static int validate(const cnsf_geometry_desc *d)
{
    if (!d) return CNSF_ERR_INVALID;
    if (d->n_x < 1 || d->n_y < 1 || d->n_views < 1 || d->n_det < 1) return CNSF_ERR_INVALID;
    if (d->n_x > (1 << 16) || d->n_y > (1 << 16) || d->n_det > (1 << 20) || d->n_views > (1 << 20))
        return CNSF_ERR_INVALID;
    if (!(d->pixel_mm > 0) || !(d->det_spacing_mm > 0) || !(d->det_width_mm > 0)) return CNSF_ERR_INVALID;
    // rays and pixels are indexed with 32-bit integers in the kernels
    if ((long long)d->n_views * d->n_det >= (1LL << 31) || (long long)d->n_x * d->n_y >= (1LL << 31))
        return CNSF_ERR_UNSUPPORTED;
    if (!std::isfinite(d->center_x_mm) || !std::isfinite(d->center_y_mm) || !std::isfinite(d->det_offset_mm))
        return CNSF_ERR_INVALID;
    if (d->detector != CNSF_DETECTOR_FLAT && d->detector != CNSF_DETECTOR_ARC &&
        d->detector != CNSF_DETECTOR_PARALLEL)
        return CNSF_ERR_UNSUPPORTED;
    if (d->detector != CNSF_DETECTOR_PARALLEL) {   // parallel rays have no source: d_po, d_ps unused
        if (!(d->d_po_mm > 0) || !(d->d_ps_mm > d->d_po_mm)) return CNSF_ERR_INVALID;
        double rx = std::fabs(d->center_x_mm) + 0.5 * d->n_x * d->pixel_mm;
        double ry = std::fabs(d->center_y_mm) + 0.5 * d->n_y * d->pixel_mm;
        if (std::hypot(rx, ry) + 2.0 * d->pixel_mm >= d->d_po_mm) return CNSF_ERR_INVALID;
    }
    if (d->detector == CNSF_DETECTOR_ARC) {   // every cell's ray within 80 deg of the central one
        double half = 0.5 * (d->n_det - 1) * d->det_spacing_mm + std::fabs(d->det_offset_mm) + 0.5 * d->det_width_mm;
        if (!(half < (80.0 / 180.0) * M_PI * d->d_ps_mm)) return CNSF_ERR_INVALID;
    }
    if (d->angles_rad)
        for (int k = 0; k < d->n_views; ++k)
            if (!std::isfinite(d->angles_rad[k])) return CNSF_ERR_INVALID;
    const int known = CNSF_OPT_NO_SYMMETRY | CNSF_OPT_EXACT_DIFFERENCES | CNSF_OPT_PLAIN_DIFFERENCES |
                      CNSF_OPT_NO_REFLECTION;
    if ((d->options & ~known) != 0) return CNSF_ERR_INVALID;
    if ((d->options & CNSF_OPT_EXACT_DIFFERENCES) && (d->options & CNSF_OPT_PLAIN_DIFFERENCES)) return CNSF_ERR_INVALID;
    return CNSF_OK;
}

// The quarter-turn symmetry of an acquisition: a square image centred on the rotation axis
// and views closed under a quarter turn, view k + V/4 at theta_k + pi/2.  Turning the whole
// acquisition of view k (source, detector line or arc, cells; Sec. II.A) by a quarter turn
// gives view k + V/4, and the turn maps the pixel lattice onto itself.
static bool quarter_turn_symmetric(const cnsf_geometry_desc *d)
{
    if (d->options & CNSF_OPT_NO_SYMMETRY) return false;
    if (d->n_x != d->n_y || d->center_x_mm != 0.0 || d->center_y_mm != 0.0 || d->n_views % 4 != 0) return false;
    if (!d->angles_rad) return true;   // 2 pi k / V
    const int q = d->n_views / 4;
    for (int k = 0; k + q < d->n_views; ++k) {
        const double r = std::remainder(d->angles_rad[k + q] - d->angles_rad[k] - 0.5 * M_PI, 2.0 * M_PI);
        if (!(std::fabs(r) <= 1e-12)) return false;
    }
    return true;
}

// The reflection symmetry on top of the quarter turns: a centred detector (cells mirror
// onto cells) and views closed under theta -> -theta, view (V - k) mod V at -theta_k.
// Mirroring the acquisition of view k in the x axis gives view -k with cell j at
// n_det - 1 - j and pixel (i, r) at (i, n_y - 1 - r) (Sec. II.A conventions).
static bool reflection_symmetric(const cnsf_geometry_desc *d)
{
    if (d->options & CNSF_OPT_NO_REFLECTION) return false;
    if (d->det_offset_mm != 0.0) return false;
    if (!d->angles_rad) return true;
    const int V = d->n_views;
    for (int k = 0; k < V; ++k) {
        const double r = std::remainder(d->angles_rad[(V - k) % V] + d->angles_rad[k], 2.0 * M_PI);
        if (!(std::fabs(r) <= 1e-12)) return false;
    }
    return true;
}

int build_geometry(const cnsf_geometry_desc *d, cnsf_geometry **out)
{
    if (!out) return CNSF_ERR_INVALID;
    *out = nullptr;
    int st = validate(d);
    if (st != CNSF_OK) return st;

    GeomConsts g{};
    g.nx = d->n_x; g.ny = d->n_y; g.nv = d->n_views; g.nd = d->n_det;
    g.h = d->pixel_mm; g.cx = d->center_x_mm; g.cy = d->center_y_mm;
    g.ds = d->det_spacing_mm; g.tau = d->det_width_mm; g.doff = d->det_offset_mm;
    g.par = d->detector == CNSF_DETECTOR_PARALLEL ? 1 : 0;
    g.arc = d->detector == CNSF_DETECTOR_ARC ? 1 : 0;
    g.dpo = g.par ? 0.0 : d->d_po_mm;
    g.dps = g.par ? 0.0 : d->d_ps_mm;
    g.rimg = std::hypot(std::fabs(g.cx) + 0.5 * g.nx * g.h, std::fabs(g.cy) + 0.5 * g.ny * g.h);
    g.s0 = cell_centre(g, 0);

    const int nv = g.nv, nd = g.nd;
    const size_t nr = (size_t)nv * nd;
    std::vector<double> cs(2 * (size_t)nv);
    for (int k = 0; k < nv; ++k) {
        double th = d->angles_rad ? d->angles_rad[k] : 2.0 * M_PI * k / nv;
        cs[2 * k] = std::cos(th);
        cs[2 * k + 1] = std::sin(th);
    }
    std::vector<double> celld(4 * (size_t)nd);
    double dtan_max = 0.0, smax = 0.0;
    for (int j = 0; j < nd; ++j) {
        // parallel rays: no direction change across cells and no perspective (blur tau at every depth)
        double sj = cell_centre(g, j), sg = 0.0, cg = 1.0, dt = 0.0;
        if (!g.par) cell_dir(g, sj, &sg, &cg, &dt);
        celld[4 * j] = sg; celld[4 * j + 1] = cg; celld[4 * j + 2] = dt; celld[4 * j + 3] = sj;
        dtan_max = std::max(dtan_max, dt);
        smax = std::max(smax, std::fabs(sj));
    }

    // Forward-walk tables and per-(view, cell) constants.
    std::vector<RayF> rays(nr);
    std::vector<BoxF> box(nr);
    std::vector<CellF> cellf(nd);
    for (int j = 0; j < nd; ++j) {
        const double sg = celld[4 * j], cg = celld[4 * j + 1], dtj = celld[4 * j + 2], sj = celld[4 * j + 3];
        // g1: s' per cell of (sigma - j) at unit depth, flat detector ds/L_j (parallel: ds);
        // the arc detector takes s' from the angle instead and leaves it unused
        cellf[j].g1 = (float)(g.par ? g.ds : g.arc ? 0.0 : g.ds / std::sqrt(g.dps * g.dps + sj * sj));
        cellf[j].c1 = (float)(g.par ? 0.5 * g.tau : 0.5 * cg * dtj);
        cellf[j].c2 = (float)(0.5 * sg * dtj);
        cellf[j].pad = 0.0f;
    }
    const double fx_one = 4294967296.0;  // 2^32
    const double tmax = g.dpo + g.rimg + g.h;
    int kc_max = 1;
    std::vector<double> hw_of(nr);
    for (int k = 0; k < nv; ++k) {
        for (int j = 0; j < nd; ++j) {
            size_t q = (size_t)k * nd + j;
            RayParams<double> R = make_ray_params<double>(g, cs[2 * k], cs[2 * k + 1], j);
            BoxConsts<double> bc = make_box_consts<double>(R.B, R.C, g.h);
            BoxF &V = box[q];
            V.q = (float)bc.q;
            V.piC = (float)(bc.p * bc.iC);
            V.iC = (float)bc.iC;
            V.hC = (float)(0.5 * R.C);
            double emax = g.par ? 0.5 * g.tau : tmax * 0.5 * R.dtan;
            double hw = (0.5 * (R.B + R.C) + emax) / R.B + 1e-3;
            int kc = (int)std::floor(2.0 * hw) + 1;
            kc_max = std::max(kc_max, kc);
            hw_of[q] = hw;
            // lines whose window [f - hw, f + hw] meets [0, na-1], widened by one
            int r0 = 0, r1 = R.nb - 1;
            if (std::fabs(R.g) < 1e-300) {
                if (R.f0 < -hw || R.f0 > R.na - 1 + hw) r1 = -1;
            } else {
                double ra = (-hw - R.f0) / R.g, rb = (R.na - 1 + hw - R.f0) / R.g;
                if (ra > rb) std::swap(ra, rb);
                double lo = std::max(0.0, std::ceil(ra) - 1.0), hi = std::min((double)(R.nb - 1), std::floor(rb) + 1.0);
                r0 = (int)lo;
                r1 = hi < lo ? -1 : (int)hi;
            }
            RayF &F = rays[q];
            F.G = std::llround(R.g * fx_one);
            F.kc = kc;
            F.flags = R.transposed;
            F.hw = (float)hw;
            F.kap = (float)R.kap;
            F.de = (float)R.de;
            // exact integer check of the candidate window at a line
            auto meets = [&](int rbi, long long A0, int r0i) {
                long long A = A0 + (long long)(rbi - r0i) * F.G;
                long long ilo = ceil_fx(A);
                return ilo <= R.na - 1 && ilo + kc - 1 >= 0;
            };
            auto a0_at = [&](int rbi) { return std::llround((R.f0 + rbi * R.g - hw) * fx_one); };
            while (r0 <= r1 && !meets(r0, a0_at(r0), r0)) ++r0;
            if (r0 <= r1) {
                long long A0 = a0_at(r0);
                while (r1 >= r0 && !meets(r1, A0, r0)) --r1;
                F.A0 = A0;
            } else {
                F.A0 = 0;
            }
            F.r0 = r0 <= r1 ? r0 : 0;
            F.nrows = r0 <= r1 ? r1 - r0 + 1 : 0;
            // Pixels of the image lie in front of the source (validated), so their depth and e
            // are positive; candidates in the zero padding may not be, but carry weight 0.
            F.e0 = (float)(R.e0 + F.r0 * R.de);
        }
    }
    // cell pairs for the back projector, in both alignments: pair m of parity o holds cells
    // 2m + o and 2m + o + 1 (a cell past n_det repeats the last cell's constants; its
    // sinogram value is 0)
    const int ndh = (nd + 1) / 2;
    // 32 bytes per cell pair (read with one 256-bit load): trapezoid constants
    // (q, q, p/C, p/C, 1/C, 1/C, -C/2, -C/2) per (parity, view, pair); cell slopes
    // (ds/L, ds/L, c1, c1, c2, c2, 0, 0) per (parity, pair)
    const size_t npairs = (size_t)nv * ndh;
    std::vector<float> box2(2 * 8 * npairs);
    std::vector<float> cell2(2 * 8 * (size_t)ndh, 0.0f);
    for (int o = 0; o < 2; ++o)
        for (int k = 0; k < nv; ++k)
            for (int m = 0; m < ndh; ++m) {
                float *A = &box2[8 * (o * npairs + (size_t)k * ndh + m)];
                for (int h = 0; h < 2; ++h) {
                    const BoxF &b = box[(size_t)k * nd + std::min(2 * m + o + h, nd - 1)];
                    A[h] = b.q; A[2 + h] = b.piC; A[4 + h] = b.iC; A[6 + h] = -b.hC;
                }
            }
    for (int o = 0; o < 2; ++o)
        for (int m = 0; m < ndh; ++m)
            for (int h = 0; h < 2; ++h) {
                const CellF &c = cellf[std::min(2 * m + o + h, nd - 1)];
                float *S = &cell2[8 * ((size_t)o * ndh + m)];
                S[h] = c.g1;
                S[2 + h] = c.c1;
                S[4 + h] = c.c2;
            }
    // The symmetric back projectors' pair table for views v < V/4 (built below when the
    // symmetry holds): per (parity, view, pair) one 32-byte entry of cells 2m + o, 2m + o + 1
    // in units of the cell's C (q/C, q'/C', p/C, p'/C', ds/(L C), ds'/(L' C'), c1/C,
    // c1'/C'; arc detector 1/C, 1/C' in the slope slots and zeros in the last two); the blur
    // needs no c2 there (c2 = c1 s_j / D_ps).
    std::vector<float> ac;
    int pad = ((kc_max + 1 + 3) / 4) * 4;
    // The walk never leaves [-pad, na-1+pad]: windows that meet [0, na-1] are at most kc wide.
    for (size_t q = 0; q < nr; ++q) {
        const RayF &F = rays[q];
        if (F.nrows == 0) continue;
        int na = F.flags ? g.ny : g.nx;
        for (int end = 0; end < 2; ++end) {
            long long A = F.A0 + (long long)(end ? F.nrows - 1 : 0) * F.G;
            long long ilo = ceil_fx(A);
            if (ilo < -pad || ilo + F.kc - 1 > na - 1 + pad) return CNSF_ERR_INTERNAL;
        }
    }

    // Launch orders.  Forward: blocks of 128 consecutive rays (the eight-value walk: blocks
    // of FP8_VT base views x FP8_CT cells) by descending walk length (lines x candidates).
    // Back: 16 x 16 tiles by descending mean magnification of their centre over the views,
    // 1/sqrt(D_po^2 - rho^2) for a tile at radius rho.
    const bool sym = quarter_turn_symmetric(d);
    const bool sym8 = sym && reflection_symmetric(d);
    if (sym) {
        const size_t np4 = (size_t)(nv / 4) * ndh;
        ac.assign(2 * 8 * np4, 0.0f);
        for (int o = 0; o < 2; ++o)
            for (int k = 0; k < nv / 4; ++k)
                for (int m = 0; m < ndh; ++m) {
                    float *A = &ac[8 * (o * np4 + (size_t)k * ndh + m)];
                    for (int hh = 0; hh < 2; ++hh) {
                        const int j = std::min(2 * m + o + hh, nd - 1);
                        const BoxF &b = box[(size_t)k * nd + j];
                        // in units of the cell's C (bp_pair_rot4): q/C, p/C, ds/(L C), c1/C; arc
                        // detector q/C, p/C, 1/C
                        const double iC = b.iC;
                        A[hh] = (float)(b.q * iC);
                        A[2 + hh] = b.piC;
                        A[4 + hh] = g.arc ? b.iC : (float)(cellf[j].g1 * iC);
                        A[6 + hh] = g.arc ? 0.0f : (float)(cellf[j].c1 * iC);
                    }
                }
    }
    const size_t nr4 = sym ? (size_t)(nv / 4) * nd : 0;
    std::vector<int> fp_order((nr + 127) / 128), fp_order4((nr4 + 127) / 128), fp_order8(sym8 ? fp8_blocks(nv, nd) : 0),
        bp_order;
    {
        auto order_blocks = [&](size_t nrays, std::vector<int> &order) {
            std::vector<std::pair<double, int>> w(order.size());
            for (size_t bi = 0; bi < order.size(); ++bi) {
                double s = 0.0;
                for (size_t q = bi * 128; q < std::min(nrays, bi * 128 + 128); ++q) s += (double)rays[q].nrows * rays[q].kc;
                w[bi] = {-s, (int)bi};
            }
            std::stable_sort(w.begin(), w.end());
            for (size_t bi = 0; bi < w.size(); ++bi) order[bi] = w[bi].second;
        };
        order_blocks(nr, fp_order);
        order_blocks(nr4, fp_order4);
        {   // the eight-value walk's blocks of FP8_VT views x FP8_CT cells
            const int nk = nv / 8 + 1, ntc = sym8 ? fp8_cell_tiles(nd) : 1;
            std::vector<std::pair<double, int>> w(fp_order8.size());
            for (size_t bi = 0; bi < w.size(); ++bi) {
                const int k0 = (int)(bi / ntc) * FP8_VT, j0 = (int)(bi % ntc) * FP8_CT;
                double s = 0.0;
                for (int k = k0; k < std::min(nk, k0 + FP8_VT); ++k)
                    for (int j = j0; j < std::min(nd, j0 + FP8_CT); ++j)
                        s += (double)rays[(size_t)k * nd + j].nrows * rays[(size_t)k * nd + j].kc;
                w[bi] = {-s, (int)bi};
            }
            std::stable_sort(w.begin(), w.end());
            for (size_t bi = 0; bi < w.size(); ++bi) fp_order8[bi] = w[bi].second;
        }
        const int tx = (g.nx + 15) / 16, ty = (g.ny + 15) / 16;
        std::vector<std::pair<double, int>> t((size_t)tx * ty);
        for (int b = 0; b < ty; ++b)
            for (int a = 0; a < tx; ++a) {
                double x = g.cx + (16.0 * a + 7.5 - 0.5 * (g.nx - 1)) * g.h;
                double y = g.cy + (16.0 * b + 7.5 - 0.5 * (g.ny - 1)) * g.h;
                double r2 = std::min(x * x + y * y, 0.99 * g.dpo * g.dpo);
                // parallel rays: every tile has the same work per view
                t[(size_t)b * tx + a] = {g.par ? 0.0 : -1.0 / std::sqrt(g.dpo * g.dpo - r2), b * tx + a};
            }
        std::stable_sort(t.begin(), t.end());
        bp_order.resize(t.size());
        for (size_t i = 0; i < t.size(); ++i) bp_order[i] = t[i].second;
    }

    cnsf_geometry *geo = new (std::nothrow) cnsf_geometry();
    if (!geo) return CNSF_ERR_NOMEM;
    geo->gc = g;
    geo->pad = pad;
    geo->kc_max = kc_max;
    geo->sym = sym ? 1 : 0;
    geo->sym8 = sym8 ? 1 : 0;
    // Window differences: the plain form loses about log2(B / tau') bits (B <= h); take the
    // exact form when the thinnest effective blur of any entry -- the cell seen at the depth of
    // the image point nearest the source (Eq. 17), tau itself for parallel rays -- falls below
    // h/32, unless the caller chose.
    {
        double dtan_min = 1e300;
        for (int j = 0; j < nd; ++j) dtan_min = std::min(dtan_min, celld[4 * j + 2]);
        const double tau_min = g.par ? g.tau : std::max(g.dpo - g.rimg, 0.0) * dtan_min;
        geo->exact = (d->options & CNSF_OPT_EXACT_DIFFERENCES) ? 1
                     : (d->options & CNSF_OPT_PLAIN_DIFFERENCES) ? 0
                                                                 : (tau_min < g.h / 32.0 ? 1 : 0);
    }
    // Back-projector window: cells within kz*zs/D_n^2*(1.02 + 2h/D_n) + ke of the pixel's
    // projection.  W bounds |s_n - s_j| over the window (widest at the nearest pixel depth).
    if (g.par) {
        // s' = ds (sigma - j); the support of M_[B, C, tau] is |s'| < (B + C + tau)/2 and B + C <= sqrt(2) h
        geo->bw.kz = 0.0;
        geo->bw.ke = (std::sqrt(2.0) * g.h + g.tau) / (2.0 * g.ds) * 1.001 + 1e-3;
    } else if (g.arc) {
        // Window in cells of D_ps/ds per radian: the footprint term as for the flat detector
        // (the pixel's distance from the source is at least its depth D_n) and the blur term
        // tau'_j/(2 R) <= dtan/2 rad, with 1% slack for the sine of the angles.
        geo->bw.kz = g.dps / (2.0 * g.ds);
        geo->bw.ke = 0.5 * dtan_max * g.dps / g.ds * 1.01 + 1e-3;
    } else {
        double dmin = g.dpo - g.rimg;
        double lmax = std::sqrt(g.dps * g.dps + (smax + g.ds) * (smax + g.ds));
        double reach = 0.5 * (std::sqrt(2.0) * g.h + tmax * dtan_max);
        double W = std::max(64.0 * g.ds, 1.5 * reach * lmax / dmin + 2.0 * g.ds);
        double ke = 0.0;
        for (int j = 0; j < nd; ++j) {
            double dt = celld[4 * j + 2], sj = celld[4 * j + 3], L = std::sqrt(g.dps * g.dps + sj * sj);
            ke = std::max(ke, (L * L / g.dps) * dt / (2.0 * g.ds) * (1.0 + std::fabs(sj) * W / (L * L)));
        }
        geo->bw.kz = g.dps / (2.0 * g.ds);
        geo->bw.ke = ke * 1.001 + 1e-3;
    }
    if (cudaGetDevice(&geo->device) != cudaSuccess) { delete geo; return record_cuda_error(); }

    struct Up { void **dst; const void *src; size_t bytes; };
    Up ups[] = {
        {(void **)&geo->d_view_cs, cs.data(), cs.size() * sizeof(double)},
        {(void **)&geo->d_cell_d, celld.data(), celld.size() * sizeof(double)},
        {(void **)&geo->d_box, box.data(), box.size() * sizeof(BoxF)},
        {(void **)&geo->d_cellf, cellf.data(), cellf.size() * sizeof(CellF)},
        {(void **)&geo->d_box2, box2.data(), box2.size() * sizeof(float)},
        {(void **)&geo->d_cell2, cell2.data(), cell2.size() * sizeof(float)},
        {(void **)&geo->d_ray, rays.data(), rays.size() * sizeof(RayF)},
        {(void **)&geo->d_fp_order, fp_order.data(), fp_order.size() * sizeof(int)},
        {(void **)&geo->d_bp_order, bp_order.data(), bp_order.size() * sizeof(int)},
        {(void **)&geo->d_fp_order4, fp_order4.data(), fp_order4.size() * sizeof(int)},
        {(void **)&geo->d_fp_order8, fp_order8.data(), fp_order8.size() * sizeof(int)},
        {(void **)&geo->d_ac, ac.data(), ac.size() * sizeof(float)},
    };
    for (const Up &u : ups) {
        if (u.bytes == 0) continue;
        cudaError_t e = cudaMalloc(u.dst, u.bytes);
        if (e != cudaSuccess) {
            destroy_geometry(geo);
            return e == cudaErrorMemoryAllocation ? (record_cuda_error(e), CNSF_ERR_NOMEM) : record_cuda_error(e);
        }
        e = cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { destroy_geometry(geo); return record_cuda_error(e); }
        geo->device_bytes += u.bytes;
    }
    st = build_tile_view_table(geo);
    if (st != CNSF_OK) { destroy_geometry(geo); return st; }
    *out = geo;
    return CNSF_OK;
}

void destroy_geometry(cnsf_geometry *geo)
{
    if (!geo) return;
    void *ptrs[] = {geo->d_view_cs, geo->d_cell_d, geo->d_box, geo->d_cellf, geo->d_ray,
                    geo->d_fp_order, geo->d_bp_order, geo->d_box2, geo->d_cell2, geo->d_tv, geo->d_tj,
                    geo->d_fp_order4, geo->d_ac, geo->d_fp_order8};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete geo;
}

}  // namespace cnsf
