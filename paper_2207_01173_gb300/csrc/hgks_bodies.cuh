// hgks_bodies.cuh -- the arithmetic of one interface position of each sweep
// pass, as templates on the scalar type and on load/store functors.  The CUDA
// kernels instantiate them with double and global-memory accessors; the host
// flop model instantiates the same bodies with an operation-counting type.
#pragma once
#include "hgks_device.cuh"
#include "hgks_kernels.cuh"

namespace hgks {

// normal reconstruction of one face (arXiv 2207.01173 Sec. 2, WENO of the cell
// averages along the face normal).  load(c, m): rotated component c of the
// m-th cell of the six along the normal (cells f-3 .. f+2).  Stores 30 slots:
// 0-4 Ql, 5-9 Qr, 10-14 dQl, 15-19 dQr, 20-24 Q0 (compatibility), 25-29 dQ0,
// slopes in index units.
template <typename T, typename Load, typename Store>
HGKS_HD void normal_body(Load load, Store store, double K)
{
    T Ql[5], Qr[5];
#pragma unroll
    for (int c = 0; c < 5; c++) {
        T X[6];
#pragma unroll
        for (int m = 0; m < 6; m++) X[m] = load(c, m);
        WenoPrep<T> wl, wr;
        weno_prep(X, wl);      // cell f-1
        weno_prep(X + 1, wr);  // cell f
        T lm_l, lm_r, r_l, r_r;
        weno_edge_pair(wl, lm_l, lm_r);
        weno_edge_pair(wr, r_l, r_r);
        Ql[c] = lm_r;
        Qr[c] = r_l;
        store(0 * 5 + c, lm_r);
        store(1 * 5 + c, r_l);
        // parabola through (left edge, average, right edge) of a cell, slope at its ends
        store(2 * 5 + c, T(2.0) * lm_l + T(4.0) * lm_r - T(6.0) * X[2]);
        store(3 * 5 + c, T(-4.0) * r_l - T(2.0) * r_r + T(6.0) * X[3]);
        // cubic through four averages, slope at the face
        store(5 * 5 + c, (T(15.0) * (X[3] - X[2]) - (X[4] - X[1])) * T(1.0 / 12.0));
    }
    // face-averaged equilibrium from the compatibility condition
    Prim<T> gl = prim_of(Ql, K), gr = prim_of(Qr, K);
    T il = T(0.5) / gl.lam, ir = T(0.5) / gr.lam;
    T ulp[3], vl[3], wl[3], urn[3], vr[3], wr[3];
    mom_half<3>(gl.U, gl.lam, il, true, ulp);
    mom_full<3>(gl.V, il, vl);
    mom_full<3>(gl.W, il, wl);
    mom_half<3>(gr.U, gr.lam, ir, false, urn);
    mom_full<3>(gr.V, ir, vr);
    mom_full<3>(gr.W, ir, wr);
    Mom<T> Ml{ ulp, vl, wl, T(K) * il, T(0.0) }, Mr{ urn, vr, wr, T(K) * ir, T(0.0) };
    T a[5], b[5];
    psi_mom<0, 0, 0>(Ml, a);
    psi_mom<0, 0, 0>(Mr, b);
#pragma unroll
    for (int c = 0; c < 5; c++) store(4 * 5 + c, gl.rho * a[c] + gr.rho * b[c]);
}

// first tangential direction of one face row.  load(slot, j): normal-pass slot
// at tangential offset j - 2.  Stores 110 slots: for Gauss line m (0, 1) at
// m*55: 25 WENO-Z values (Ql, Qr, dQl, dQr, dQ0), 15 quartic values and 15
// quartic derivatives (Ql, Qr, Q0).
template <typename T, typename Load, typename Store>
HGKS_HD void tan1_body(Load load, Store store)
{
#pragma unroll 1
    for (int w = 0; w < 5; w++) {
        const int slot = w < 4 ? w : 5;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            T X[5];
#pragma unroll
            for (int j = 0; j < 5; j++) X[j] = load(slot * 5 + c, j);
            WenoPrep<T> W;
            weno_prep(X, W);
            T vm, vp;
            weno_gauss_pair(W, vm, vp);
            store(0 * 55 + w * 5 + c, vm);
            store(1 * 55 + w * 5 + c, vp);
        }
    }
#pragma unroll 1
    for (int l = 0; l < 3; l++) {
        const int slot = l < 2 ? l : 4;
#pragma unroll
        for (int c = 0; c < 5; c++) {
            T X[5];
#pragma unroll
            for (int j = 0; j < 5; j++) X[j] = load(slot * 5 + c, j);
            T vm, vp, dm, dp;
            quartic_value_pair(X, vm, vp);
            quartic_deriv_pair(X, dm, dp);
            store(0 * 55 + 25 + l * 5 + c, vm);
            store(1 * 55 + 25 + l * 5 + c, vp);
            store(0 * 55 + 40 + l * 5 + c, dm);
            store(1 * 55 + 40 + l * 5 + c, dp);
        }
    }
}

// geometry of one face: inverse normal metric, inverse tangential metrics at
// the Gauss abscissae, area
struct FaceGeom {
    double ihn, ih1[2], ih2[2], area;
};

// the geometry of face f of sweep d (between cells f-1 and f along d) at
// tangential cell indices (a, b): y metrics from the Params tables (dy/dj at
// the faces and at the Gauss abscissae), uniform spacings elsewhere; the
// face area uses the cell height of its y row
HGKS_HD FaceGeom face_geom(const Params &P, int d, int f, int a, int b)
{
    const int e1 = tdir(d, 0), e2 = tdir(d, 1);
    FaceGeom G;
    G.ihn = 1.0 / (d == 1 ? P.my_face[f] : P.h[d]);
    if (d == 0) G.area = P.hy_cell[a] * P.h[2];
    else if (d == 1) G.area = P.h[0] * P.h[2];
    else G.area = P.h[0] * P.hy_cell[b];
    for (int m = 0; m < 2; m++) {
        G.ih1[m] = 1.0 / (e1 == 1 ? P.my_gp[2 * a + m] : P.h[e1]);
        G.ih2[m] = 1.0 / (e2 == 1 ? P.my_gp[2 * b + m] : P.h[e2]);
    }
    return G;
}

// second tangential direction, the four Gauss-point fluxes and their sum.
// load(slot, j): first-pass slot at offset j - 2 along the second tangential
// direction.  col: scratch of 110 values for the inputs of the two Gauss
// points of a line, laid out as the point flux reads them: for Gauss point n
// at n * 55: Ql (5), Qr (5), then the physical slopes dl[3][5], dr[3][5],
// d0[3][5] (normal, t1, t2).  Fs, dFs: F^n and dF^n/dt times the face area,
// rotated frame.
template <typename T, typename Load>
HGKS_HD void flux_body(Load load, const FaceGeom &G, const Params &P, T dt, T *col, T Fs[5], T dFs[5])
{
#pragma unroll
    for (int c = 0; c < 5; c++) {
        Fs[c] = T(0.0);
        dFs[c] = T(0.0);
    }
#pragma unroll 1
    for (int m = 0; m < 2; m++) {
        const double ih1 = G.ih1[m];
        // WENO to the Gauss points: values of Ql, Qr (rows 0..9), normal slopes (rows 10..24)
#pragma unroll 1
        for (int k = 0; k < 25; k++) {
            T X[5];
#pragma unroll
            for (int j = 0; j < 5; j++) X[j] = load(m * 55 + k, j);
            WenoPrep<T> W;
            weno_prep(X, W);
            T v0, v1;
            weno_gauss_pair(W, v0, v1);
            if (k < 10) {
                col[k] = v0;
                col[55 + k] = v1;
            } else {
                const int slot = k < 15 ? k : (k < 20 ? k + 10 : k + 20);  // dl/dr/d0[0][c]
                col[slot] = v0 * T(G.ihn);
                col[55 + slot] = v1 * T(G.ihn);
            }
        }
        // first-direction derivatives (quartic value) and second-direction derivatives
        // of the first-direction quartic values (quartic derivative)
#pragma unroll 1
        for (int k = 0; k < 15; k++) {
            T X[5], Y[5];
#pragma unroll
            for (int j = 0; j < 5; j++) {
                X[j] = load(m * 55 + 40 + k, j);
                Y[j] = load(m * 55 + 25 + k, j);
            }
            T a0, a1, b0, b1;
            quartic_value_pair(X, a0, a1);
            quartic_deriv_pair(Y, b0, b1);
            const int slot = 10 + (k / 5) * 15 + k % 5;  // d[.][0][c] of state k / 5
            col[slot + 5] = a0 * T(ih1);
            col[55 + slot + 5] = a1 * T(ih1);
            col[slot + 10] = b0 * T(G.ih2[0]);
            col[55 + slot + 10] = b1 * T(G.ih2[1]);
        }
#pragma unroll 1
        for (int n = 0; n < 2; n++) {
            const T *g = col + 55 * n;
            T Fn[5], dFn[5];
            gks_point_flux<T>(g, g + 5, (const T(*)[5])(g + 10), (const T(*)[5])(g + 25), (const T(*)[5])(g + 40), P,
                              dt, Fn, dFn);
#pragma unroll
            for (int c = 0; c < 5; c++) {
                Fs[c] += T(0.25) * Fn[c];
                dFs[c] += T(0.25) * dFn[c];
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 5; c++) {
        Fs[c] = Fs[c] * T(G.area);
        dFs[c] = dFs[c] * T(G.area);
    }
}

}  // namespace hgks
