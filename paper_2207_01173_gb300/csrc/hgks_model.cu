// hgks_model.cu -- algorithmic floating-point work of one HGKS step.
//
// The kernels' arithmetic lives in templates (hgks_device.cuh,
// hgks_bodies.cuh).  Here the same templates run on the host with an
// operation-counting scalar, so the count follows the code that runs on the
// GPU.  Counting rule: +, -, * count 1 each (a fused a*b+c counts 2);
// division, sqrt, exp, erfc and pow count 1 each and are also reported on
// their own; index arithmetic, comparisons, sign changes and fabs count 0.
#include "../../include/hgks.h"
#include "hgks_bodies.cuh"
#include "hgks_kernels.cuh"

#include <cmath>

namespace hgks_count {

struct Tally {
    double add = 0, mul = 0, div = 0, special = 0;
    double flops() const { return add + mul + div + special; }
};
static Tally *cur = nullptr;

struct Num {
    double v;
    Num() : v(0.0) {}
    Num(double x) : v(x) {}
};
inline Num operator+(Num a, Num b) { cur->add += 1; return Num(a.v + b.v); }
inline Num operator-(Num a, Num b) { cur->add += 1; return Num(a.v - b.v); }
inline Num operator*(Num a, Num b) { cur->mul += 1; return Num(a.v * b.v); }
inline Num operator/(Num a, Num b) { cur->div += 1; return Num(a.v / b.v); }
inline Num operator-(Num a) { return Num(-a.v); }
inline Num &operator+=(Num &a, Num b) { a = a + b; return a; }
inline Num &operator-=(Num &a, Num b) { a = a - b; return a; }
inline Num &operator*=(Num &a, Num b) { a = a * b; return a; }
inline bool operator>(Num a, Num b) { return a.v > b.v; }
inline bool operator<(Num a, Num b) { return a.v < b.v; }
inline Num fabs(Num a) { return Num(std::fabs(a.v)); }
inline Num sqrt(Num a) { cur->special += 1; return Num(std::sqrt(a.v)); }
inline Num exp(Num a) { cur->special += 1; return Num(std::exp(a.v)); }
inline Num erfc(Num a) { cur->special += 1; return Num(std::erfc(a.v)); }
inline Num pow(Num a, Num e) { cur->special += 1; return Num(std::pow(a.v, e.v)); }

}  // namespace hgks_count

using hgks_count::Num;
using hgks_count::Tally;

// a smooth, physically valid sample state for the bodies (the count does not
// depend on the values: the only data-dependent branch, tau > 0, is taken)
static double sample(int slot, int j)
{
    const double base[5] = { 1.0, 0.3, -0.2, 0.1, 180.0 };
    return base[slot % 5] * (1.0 + 1e-3 * (slot % 7) + 1e-4 * j);
}

extern "C" hgks_status hgks_flop_model(const hgks_grid *grid, hgks_precision precision, hgks_flop_model_t *out)
{
    if (!grid || !out || grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return HGKS_ERR_INVALID_ARG;
    if (precision != HGKS_FP64) return HGKS_ERR_INVALID_ARG;
    using namespace hgks;
    Params P;
    memset(&P, 0, sizeof P);
    P.gamma = 1.4;
    P.K = 2.0;
    P.Pr = 0.72;
    P.visc_kind = 1;
    P.mu_ref = 1e-3;
    P.T_ref = 70.0;
    P.omega = 0.7;

    Tally tn, tt, tf;
    // normal pass, one face
    hgks_count::cur = &tn;
    {
        auto load = [](int c, int m) { return Num(c == 4 ? 180.0 + 0.01 * m : (c == 0 ? 1.0 + 0.001 * m : 0.1 * c + 0.01 * m)); };
        auto store = [](int, Num) {};
        normal_body<Num>(load, store, P.K);
    }
    // first tangential pass, one position
    hgks_count::cur = &tt;
    {
        auto load = [](int slot, int j) { return Num(sample(slot, j)); };
        auto store = [](int, Num) {};
        tan1_body<Num>(load, store);
    }
    // flux pass, one face
    hgks_count::cur = &tf;
    {
        // slots 0-4 Ql, 5-9 Qr (valid states), 10-24 normal slopes, 25-54 quartic values/derivatives
        auto load = [](int slot, int j) {
            int s = slot % 55;
            if (s < 10 || (s >= 25 && s < 40)) return Num(sample(s % 5, j));
            return Num(1e-2 * (1 + s % 5) + 1e-3 * j);
        };
        FaceGeom G;
        G.ihn = 50.0;
        G.ih1[0] = G.ih1[1] = G.ih2[0] = G.ih2[1] = 50.0;
        G.area = 4e-4;
        Num Fs[5], dFs[5], col[110];
        flux_body<Num>(load, G, P, Num(1e-3), col, Fs, dFs);
    }
    hgks_count::cur = nullptr;

    Params S;
    memset(&S, 0, sizeof S);
    S.n[0] = grid->nx;
    S.n[1] = grid->ny;
    S.n[2] = grid->nz;
    double per_stage = 0.0;
    for (int d = 0; d < 3; d++)
        per_stage += (double)box_count(box_fq(S, d)) * tn.flops() + (double)box_count(box_t1(S, d)) * tt.flops() +
                     (double)box_count(box_face(S, d)) * tf.flops();
    const double cells = (double)grid->nx * grid->ny * grid->nz;
    // per cell and stage: flux divergence 2 x 5 x (3 differences + 2 adds + 1 division),
    // stage update about 2 x 5 x 3; the CFL reduction about 20 per cell once per step
    const double update = 2.0 * 5.0 * 6.0 + 30.0;
    out->normal_per_face = tn.flops();
    out->tan1_per_pos = tt.flops();
    out->flux_per_face = tf.flops();
    out->div_per_face_flux = tf.div;
    out->special_per_face_flux = tf.special;
    out->per_step = 2.0 * (per_stage + cells * update) + 20.0 * cells;
    return HGKS_OK;
}
