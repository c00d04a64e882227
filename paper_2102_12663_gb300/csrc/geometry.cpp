// Host-side geometry: the analytic eye of the anterior segment and the
// validation of caller-supplied masks (arXiv 2102.12663, Sec. 2.1, Tab. 1).
//
// The paper's Fig. 1 is not part of its text and Tab. 1's dimensions do not fit
// a 2:1 lattice, so the eye is this library's own construction:
//   * cell centres at integer (x, y); x across the chamber, y along the
//     optical axis, lens/iris at the bottom;
//   * solid outer ring (adiabatic walls);
//   * iris/lens band y < band (hot wall Gamma_2) between the two angle points
//     xa and nx-1-xa; outside them the band is sclera (adiabatic);
//   * ciliary-body inlet: the band's top row over a centred gap of inlet_w
//     cells, parabolic inflow along +y;
//   * cornea (cold wall Gamma_1): everything above the band outside a circular
//     arc that spans the chord y = band - 1/2 between (xa - 1/2) and
//     (nx - 1 - xa + 1/2); its sagitta h = a tan(alpha/2) (a = half chord)
//     makes the arc meet the iris plane at the chamber angle alpha;
//   * trabecular meshwork (Omega_3): the part outside the arc of a box
//     [xa - tm_w, xa + tm_w) x [band, band + tm_h) at each angle, porous, with
//     a one-cell outlet column (Schlemm's canal side) at x = xa - tm_w - 1.
// Defaults scale the 160 x 80 reference eye: band ny/10, inlet 4 and TM
// 6 x 10 cells per 160 columns.  Mirror-symmetric about x = (nx - 1)/2.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"

namespace lbm {

static int iround(double v) { return (int)std::floor(v + 0.5); }

static bool eye_mask(const lbm_geometry_desc& g, uint8_t* out, lbm_geometry_info* info,
                     std::string& err) {
    const int nx = g.nx, ny = g.ny;
    const double alpha = g.chamber_angle_deg;
    if (nx < 16 || ny < 8) { err = "eye needs nx >= 16 and ny >= 8"; return false; }
    if (!(alpha > 0.0 && alpha < 180.0)) { err = "chamber angle must lie in (0, 180) degrees"; return false; }
    int band = g.band_cells > 0 ? g.band_cells : iround(ny / 10.0);
    int w_in = g.inlet_cells > 0 ? g.inlet_cells : std::max(2, iround(4.0 * nx / 160.0));
    if ((nx - w_in) % 2 != 0) w_in += 1;  // keep the gap centred on the mirror axis
    const int tw = g.tm_w > 0 ? g.tm_w : std::max(2, iround(6.0 * nx / 160.0));
    const int th = g.tm_h > 0 ? g.tm_h : std::max(2, iround(10.0 * nx / 160.0));
    const int xa = tw + 2;
    const double half_chord = 0.5 * nx - xa;
    const double x_mid = 0.5 * (nx - 1);
    const double y_chord = band - 0.5;
    const double sag = half_chord * std::tan(alpha * M_PI / 360.0);
    const double R = (half_chord * half_chord + sag * sag) / (2.0 * sag);
    const double y_ctr = y_chord + sag - R;
    const int gap0 = (nx - w_in) / 2;
    if (band < 2 || half_chord <= tw + 1 || y_chord + sag >= ny - 1.5 || band + th >= ny - 1 ||
        w_in >= 2 * half_chord - 2) {
        err = "eye geometry does not fit the grid (angle too wide or grid too small)";
        return false;
    }
    if (out) {
        for (int y = 0; y < ny; ++y) {
            uint8_t* row = out + (int64_t)y * nx;
            for (int x = 0; x < nx; ++x) {
                const int xs = std::min(x, nx - 1 - x);  // distance from the nearer side
                uint8_t t;
                if (x == 0 || y == 0 || x == nx - 1 || y == ny - 1) {
                    t = LBM_CELL_ADIABATIC;
                } else if (y < band) {
                    const bool gap = y == band - 1 && x >= gap0 && x < gap0 + w_in;
                    t = gap ? LBM_CELL_INLET : (xs >= xa ? LBM_CELL_HOT : LBM_CELL_ADIABATIC);
                } else {
                    const double dx = x - x_mid, dy = y - y_ctr;
                    const bool tm_rows = y < band + th;
                    if (dx * dx + dy * dy < R * R) t = LBM_CELL_FLUID;
                    else if (tm_rows && xs >= xa - tw && xs < xa + tw) t = LBM_CELL_POROUS;
                    else if (tm_rows && xs == xa - tw - 1) t = LBM_CELL_OUTLET;
                    else t = xs >= xa ? LBM_CELL_COLD : LBM_CELL_ADIABATIC;
                }
                row[x] = t;
            }
        }
    }
    if (info) {
        info->inlet_dir_x = 0;
        info->inlet_dir_y = 1;
        info->inlet_profile = 1;
        info->inlet_lo = gap0;
        info->inlet_width = w_in;
        info->eye_normals = 1;
        info->outlet_axis = 0;
        info->arc_xc = x_mid;
        info->arc_yc = y_ctr;
        info->arc_r = R;
    }
    return true;
}

// Builds the mask of `g` into out (may be null) and fills info.  Returns false
// with a message in err when the description is invalid.
bool build_mask(const lbm_geometry_desc& g, uint8_t* out, lbm_geometry_info* info,
                std::string& err) {
    if (g.nx <= 0 || g.ny <= 0 || (int64_t)g.nx * g.ny > (int64_t)1 << 30) {
        err = "grid size out of range";
        return false;
    }
    lbm_geometry_info tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    std::vector<uint8_t> own;
    const int64_t N = (int64_t)g.nx * g.ny;
    if (!out) {
        own.resize(N);
        out = own.data();
    }
    bool periodic_x = false, periodic_y = false;
    if (g.kind == LBM_GEOM_EYE) {
        if (!eye_mask(g, out, &tmp, err)) return false;
    } else if (g.kind == LBM_GEOM_MASK) {
        if (!g.host_mask) { err = "MASK geometry without host_mask"; return false; }
        std::memcpy(out, g.host_mask, (size_t)N);
        periodic_x = g.periodic_x != 0;
        periodic_y = g.periodic_y != 0;
        tmp.inlet_dir_x = g.inlet_dir_x;
        tmp.inlet_dir_y = g.inlet_dir_y;
        tmp.inlet_profile = g.inlet_profile;
        tmp.inlet_lo = g.inlet_lo;
        tmp.inlet_width = g.inlet_width;
        tmp.eye_normals = 0;
        tmp.outlet_axis = g.inlet_dir_x != 0 ? 0 : 1;
    } else {
        err = "unknown geometry kind";
        return false;
    }
    tmp.n_cells = N;
    for (int y = 0; y < g.ny; ++y) {
        for (int x = 0; x < g.nx; ++x) {
            const uint8_t t = out[(int64_t)y * g.nx + x];
            if (t > LBM_CELL_OUTLET) { err = "mask holds an unknown cell type"; return false; }
            const bool active = t == LBM_CELL_FLUID || t == LBM_CELL_POROUS;
            if (active) {
                ++tmp.n_active;
                if ((!periodic_x && (x == 0 || x == g.nx - 1)) ||
                    (!periodic_y && (y == 0 || y == g.ny - 1))) {
                    err = "an active cell lies on a non-periodic edge";
                    return false;
                }
            }
            tmp.n_fluid += t == LBM_CELL_FLUID;
            tmp.n_porous += t == LBM_CELL_POROUS;
            tmp.n_inlet += t == LBM_CELL_INLET;
            tmp.n_outlet += t == LBM_CELL_OUTLET;
        }
    }
    if (tmp.n_active == 0) { err = "mask has no fluid or porous cell"; return false; }
    if (tmp.n_inlet > 0) {
        const int ax = std::abs(tmp.inlet_dir_x), ay = std::abs(tmp.inlet_dir_y);
        if (ax + ay != 1) { err = "inlet direction must be a lattice axis"; return false; }
        if (tmp.inlet_profile == 1 && tmp.inlet_width < 1) { err = "parabolic inlet needs inlet_width >= 1"; return false; }
        if (tmp.inlet_profile != 0 && tmp.inlet_profile != 1) { err = "inlet_profile must be 0 or 1"; return false; }
    }
    if (info) *info = tmp;
    return true;
}

// Sets the near-boundary bit of every active cell that has a non-active
// neighbour (periodic wrap on flagged edges).
void mark_near_boundary(uint8_t* m, int nx, int ny) {
    static const int EXv[8] = {1, 0, -1, 0, 1, -1, -1, 1};
    static const int EYv[8] = {0, 1, 0, -1, 1, 1, -1, -1};
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            uint8_t& t = m[(int64_t)y * nx + x];
            const uint8_t ty = t & 7;
            if (ty > LBM_CELL_POROUS) continue;
            bool near = false;
            for (int k = 0; k < 8 && !near; ++k) {
                const int xn = (x + EXv[k] + nx) % nx, yn = (y + EYv[k] + ny) % ny;
                const uint8_t tn = m[(int64_t)yn * nx + xn] & 7;
                near = tn > LBM_CELL_POROUS;
            }
            if (near) t |= 8;
        }
    }
}

}  // namespace lbm
