// Host/device description of an Alard-Lupton basis specification: function
// order (g, p, q), spatial and background term counts, number of unknowns.
#pragma once
#include <string.h>

#include "argus_internal.cuh"

struct BasisDev {
    int ks, r, ng, nb, NH;
    int sdeg, bgdeg, Ks, Kb, Nc;
    float sigma[ARGUS_MAX_NG];
    int hoff[ARGUS_MAX_NG];
    int g[ARGUS_MAX_NB], p[ARGUS_MAX_NB], q[ARGUS_MAX_NB];
};

inline int nterms(int d) { return d < 0 ? 0 : (d + 1) * (d + 2) / 2; }

inline int make_basis_dev(const argus_basis* b, BasisDev* d) {
    if (!b || b->ksize < 3 || b->ksize > ARGUS_MAX_KS || !(b->ksize & 1)) return ARGUS_ERR_ARG;
    if (b->ngauss < 1 || b->ngauss > ARGUS_MAX_NG) return ARGUS_ERR_ARG;
    if (b->spatial_degree < 0 || b->spatial_degree > 2 || b->bg_degree < 0 || b->bg_degree > 2)
        return ARGUS_ERR_ARG;
    memset(d, 0, sizeof(*d));
    d->ks = b->ksize;
    d->r = (b->ksize - 1) / 2;
    d->ng = b->ngauss;
    int n = 0, nh = 0;
    for (int g = 0; g < b->ngauss; g++) {
        const int deg = b->degree[g];
        if (deg < 0 || deg > 8 || !(b->sigma[g] > 0.0f)) return ARGUS_ERR_ARG;
        d->sigma[g] = b->sigma[g];
        d->hoff[g] = nh;
        nh += deg + 1;
        for (int p = 0; p <= deg; p++)
            for (int q = 0; q <= deg - p; q++) {
                if (n >= ARGUS_MAX_NB) return ARGUS_ERR_UNSUPPORTED;
                d->g[n] = g; d->p[n] = p; d->q[n] = q;
                n++;
            }
    }
    d->nb = n;
    d->NH = nh;
    d->sdeg = b->spatial_degree;
    d->bgdeg = b->bg_degree;
    d->Ks = nterms(b->spatial_degree);
    d->Kb = nterms(b->bg_degree);
    d->Nc = 1 + (n - 1) * d->Ks + d->Kb;
    return ARGUS_OK;
}
