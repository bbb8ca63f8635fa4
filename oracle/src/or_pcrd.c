/*
 * EBCC oracle (test infrastructure only): post-compression rate-distortion
 * optimisation (PCRD-opt, Taubman's EBCOT rate allocation as used by JPEG2000
 * encoders).  Algorithm 1's enc_base(A, r, eps) compresses "with a compression
 * ratio r"; reading c3: a byte budget of 4N/r for the code-block payloads.
 *
 * Per code-block: the lower convex hull of its (rate, distortion) truncation
 * points.  Across blocks: sort every hull segment by slope, highest first, and
 * take whole groups of equal slope while the running rate stays within the
 * budget.  A block keeps the hull points whose segment slope is at least the
 * last slope taken.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

void or_pcrd_hull(const or_t1_result *r, or_hull *h) {
    int np = r->npasses;
    int64_t D[OR_T1_MAXPASS + 1];
    long R[OR_T1_MAXPASS + 1];
    D[0] = r->D0; R[0] = 0;
    for (int n = 1; n <= np; n++) { D[n] = D[n - 1] - r->dD[n - 1]; R[n] = r->pass_len[n - 1]; }
    int nh = 1;
    h->pt[0] = 0; h->rate[0] = 0; h->slope[0] = INFINITY;
    for (int n = 1; n <= np; n++) {
        if (D[n] >= D[h->pt[nh - 1]]) continue;
        double s = 0;
        for (;;) {
            int last = h->pt[nh - 1];
            long dR = R[n] - R[last];
            int64_t dD = D[last] - D[n];
            if (dR <= 0) { nh--; continue; } /* last >= 1 here: R[n] >= 1 for n >= 1 */
            s = (double)dD / (double)dR;
            if (nh >= 2 && s >= h->slope[nh - 1]) { nh--; continue; }
            break;
        }
        h->pt[nh] = n; h->rate[nh] = R[n]; h->slope[nh] = s; nh++;
    }
    h->nhull = nh;
}

typedef struct { double slope; long dR; } seg;

static int seg_desc(const void *a, const void *b) {
    double x = ((const seg *)a)->slope, y = ((const seg *)b)->slope;
    return x < y ? 1 : (x > y ? -1 : 0);
}

void or_pcrd_select(const or_hull *hulls, int nb, double budget, int *np_out) {
    long nseg = 0;
    for (int b = 0; b < nb; b++) nseg += hulls[b].nhull - 1;
    seg *sg = (seg *)malloc(sizeof(seg) * (nseg + 1));
    long k = 0;
    for (int b = 0; b < nb; b++)
        for (int i = 1; i < hulls[b].nhull; i++) {
            sg[k].slope = hulls[b].slope[i];
            sg[k].dR = hulls[b].rate[i] - hulls[b].rate[i - 1];
            k++;
        }
    qsort(sg, nseg, sizeof(seg), seg_desc);
    double thr = INFINITY;
    long cum = 0;
    for (long i = 0; i < nseg;) {
        long j = i, grp = 0;
        while (j < nseg && sg[j].slope == sg[i].slope) grp += sg[j++].dR;
        if ((double)(cum + grp) > budget) break;
        cum += grp;
        thr = sg[i].slope;
        i = j;
    }
    for (int b = 0; b < nb; b++) {
        int n = 0;
        for (int i = 1; i < hulls[b].nhull; i++)
            if (hulls[b].slope[i] >= thr) n = hulls[b].pt[i];
        np_out[b] = n;
    }
    free(sg);
}
