// hgks_mesh.h -- host tables of the y mesh (arXiv 2207.01173 Sec. 4.2 map,
// y(s) = y0 + ly/2 (1 + tanh(b (s - 1)) / tanh b), s = 2 j / ny; uniform
// spacing when b = 0).  Reconstruction works in index space, and a physical
// derivative along y is the index derivative divided by dy/dj at the point
// where it is taken, so the tables hold dy/dj at the faces, at the two Gauss
// abscissae of each cell and at the cell centres, with the cell heights and
// the face and centre coordinates.
#pragma once
#include "../../include/hgks.h"

#include <cmath>
#include <cstddef>
#include <vector>

namespace hgks {

inline double mesh_y_at(const hgks_grid &g, double s)  // s = 2 j / ny in [0, 2]
{
    if (!(g.y_stretch_b > 0.0)) return g.y0 + 0.5 * s * g.ly;
    const double b = g.y_stretch_b;
    return g.y0 + 0.5 * g.ly * (1.0 + std::tanh(b * (s - 1.0)) / std::tanh(b));
}

inline double mesh_dydj_at(const hgks_grid &g, double jpos)
{
    const double ds = 2.0 / g.ny;
    if (!(g.y_stretch_b > 0.0)) return g.ly / g.ny;
    const double b = g.y_stretch_b, th = std::tanh(b * (jpos * ds - 1.0));
    return 0.5 * g.ly * b * (1.0 - th * th) / std::tanh(b) * ds;
}

// layout: my_face[ny+1] | my_gp[2 ny] | my_cen[ny] | hy_cell[ny] | yface[ny+1] | ycen[ny]
inline std::vector<double> mesh_y_tables(const hgks_grid &g)
{
    const int ny = g.ny;
    const bool st = g.y_stretch_b > 0.0;
    std::vector<double> t((size_t)(ny + 1) * 2 + (size_t)ny * 5);
    double *my_face = t.data(), *my_gp = my_face + ny + 1, *my_cen = my_gp + 2 * ny, *hy = my_cen + ny,
           *yface = hy + ny, *ycen = yface + ny + 1;
    const double g6 = std::sqrt(3.0) / 6.0;
    for (int j = 0; j <= ny; j++) {
        my_face[j] = mesh_dydj_at(g, j);
        yface[j] = st ? mesh_y_at(g, 2.0 * j / ny) : g.y0 + j * (g.ly / ny);
    }
    for (int j = 0; j < ny; j++) {
        my_gp[2 * j] = mesh_dydj_at(g, j + 0.5 - g6);
        my_gp[2 * j + 1] = mesh_dydj_at(g, j + 0.5 + g6);
        my_cen[j] = mesh_dydj_at(g, j + 0.5);
        hy[j] = st ? yface[j + 1] - yface[j] : g.ly / ny;
        ycen[j] = mesh_y_at(g, 2.0 * (j + 0.5) / ny);
    }
    return t;
}

}  // namespace hgks
