/*
 * CPU ORACLE -- test infrastructure only (per-object steps after the labels).
 *
 * Plain CPU definitions of the two steps that follow the distance transform
 * in the paper's pipeline (Teodoro et al., "Region Templates", Section 5.1
 * "Example Application"): Watershed, which splits touching nuclei after the
 * Pre-Watershed step, and the feature computation stage, which computes
 * shape and texture features of every segmented nucleus from per-nucleus
 * intermediate results (histograms and co-occurrence matrices). The paper
 * names these steps without defining them; each function states the
 * definition it computes.
 *
 * Only the test suite may load this code; it shares nothing with the CUDA
 * sources. Images are row-major and contiguous (stride W). Objects are the
 * pixels sharing one label value >= 0 of a label image L (-1 = background).
 * Return value 0 = ok, -1 = bad argument, -2 = out of memory.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NFEAT 20

static int cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* index of value v in the sorted array s[0..n-1], or -1 */
static long find_sorted(const int32_t *s, long n, int32_t v)
{
    long lo = 0, hi = n - 1;
    while (lo <= hi) {
        const long m = (lo + hi) / 2;
        if (s[m] == v) return m;
        if (s[m] < v) lo = m + 1;
        else hi = m - 1;
    }
    return -1;
}

/* The distinct label values >= 0 of L, ascending, into *out (malloc'ed);
 * returns their number or -2. */
static long distinct_labels(const int32_t *L, long N, int32_t **out)
{
    long n = 0;
    for (long p = 0; p < N; p++) n += L[p] >= 0;
    int32_t *v = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!v) return -2;
    n = 0;
    for (long p = 0; p < N; p++)
        if (L[p] >= 0) v[n++] = L[p];
    qsort(v, (size_t)n, sizeof(int32_t), cmp_i32);
    long u = 0;
    for (long i = 0; i < n; i++)
        if (u == 0 || v[i] != v[u - 1]) v[u++] = v[i];
    *out = v;
    return u;
}

/* ------------------------------------------------------- object features */
/* Feature computation stage (Section 5.1): per object, intermediate results
 * are accumulated first (pixel count, bounding box, coordinate moments,
 * perimeter, the 256-bin intensity histogram, the co-occurrence matrix), then
 * the features are computed from them. Features of an object S, in order:
 *   0 area |S|;  1 perimeter: pixel edges between S and a 4-neighbour not in
 *   S (outside the image counts as not in S);  2, 3 bounding box height and
 *   width;  4, 5 centroid row and column;  6, 7 major and minor axis lengths
 *   4 sqrt(l1), 4 sqrt(l2), l1 >= l2 the eigenvalues of the population
 *   covariance of the pixel coordinates (l2 raised to 0);  8 eccentricity
 *   sqrt(1 - l2 / l1) (0 when l1 = 0);  9 compactness 4 pi |S| / perimeter^2;
 *   10, 11 mean and population standard deviation of the intensity;  12, 13
 *   its minimum and maximum;  14 its median (the smallest v with
 *   2 #{I <= v} >= |S|);  15 the histogram's entropy in bits;  16 the
 *   number of co-occurrence pairs: horizontally adjacent pixels (r, c),
 *   (r, c + 1) both in S, with the intensities quantised to 8 levels
 *   (I >> 5); 17 contrast sum (a - b)^2 g(a,b) / n2;  18 energy
 *   sum g(a,b)^2 / n2^2;  19 homogeneity sum g(a,b) / (1 + |a - b|) / n2 (a
 *   outer, b inner; 0 for 17..19 when there is no pair).
 * Second moments are formed exactly in integers (coordinates relative to the
 * bounding box, products in 128 bits) before the one division, so that the
 * floating-point steps start from exact values. Objects are ordered by
 * label; at most cap are written, *n_obj receives their total number. */
int orc_object_features(const int32_t *L, const uint8_t *I, int H, int W, int cap, int32_t *labels,
                        double *feat, int *n_obj)
{
    if (!L || !I || H < 1 || W < 1 || cap < 0 || !n_obj) return -1;
    const long N = (long)H * W;
    int32_t *lab = NULL;
    const long n = distinct_labels(L, N, &lab);
    if (n < 0) return -2;
    *n_obj = (int)n;
    const long m = n > 0 ? n : 1;
    int64_t *area = calloc((size_t)m, 8), *per = calloc((size_t)m, 8);
    int64_t *r0 = malloc((size_t)m * 8), *c0 = malloc((size_t)m * 8), *r1 = malloc((size_t)m * 8),
            *c1 = malloc((size_t)m * 8);
    int64_t *hist = calloc((size_t)m * 256, 8), *glcm = calloc((size_t)m * 64, 8);
    if (!area || !per || !r0 || !c0 || !r1 || !c1 || !hist || !glcm) {
        free(lab); free(area); free(per); free(r0); free(c0); free(r1); free(c1); free(hist); free(glcm);
        return -2;
    }
    for (long k = 0; k < n; k++) {
        r0[k] = c0[k] = INT64_MAX;
        r1[k] = c1[k] = -1;
    }
    /* pass 1: counts, bounding boxes, perimeter, histogram, co-occurrences */
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            const int32_t l = L[(long)r * W + c];
            if (l < 0) continue;
            const long k = find_sorted(lab, n, l);
            area[k]++;
            if (r < r0[k]) r0[k] = r;
            if (r > r1[k]) r1[k] = r;
            if (c < c0[k]) c0[k] = c;
            if (c > c1[k]) c1[k] = c;
            const int dr[4] = {-1, 1, 0, 0}, dc[4] = {0, 0, -1, 1};
            for (int e = 0; e < 4; e++) {
                const int rr = r + dr[e], cc = c + dc[e];
                if (rr < 0 || rr >= H || cc < 0 || cc >= W || L[(long)rr * W + cc] != l) per[k]++;
            }
            const int v = I[(long)r * W + c];
            hist[k * 256 + v]++;
            if (c + 1 < W && L[(long)r * W + c + 1] == l) glcm[k * 64 + (v >> 5) * 8 + (I[(long)r * W + c + 1] >> 5)]++;
        }
    /* pass 2: coordinate moments relative to the bounding box */
    int64_t *sr = calloc((size_t)m, 8), *sc = calloc((size_t)m, 8), *srr = calloc((size_t)m, 8),
            *scc = calloc((size_t)m, 8), *src = calloc((size_t)m, 8);
    if (!sr || !sc || !srr || !scc || !src) {
        free(lab); free(area); free(per); free(r0); free(c0); free(r1); free(c1); free(hist); free(glcm);
        free(sr); free(sc); free(srr); free(scc); free(src);
        return -2;
    }
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            const int32_t l = L[(long)r * W + c];
            if (l < 0) continue;
            const long k = find_sorted(lab, n, l);
            const int64_t y = r - r0[k], x = c - c0[k];
            sr[k] += y;
            sc[k] += x;
            srr[k] += y * y;
            scc[k] += x * x;
            src[k] += y * x;
        }
    const long nw = n < cap ? n : cap;
    for (long k = 0; k < nw; k++) {
        double *f = feat + k * NFEAT;
        const int64_t a = area[k];
        const double da = (double)a;
        labels[k] = lab[k];
        f[0] = da;
        f[1] = (double)per[k];
        f[2] = (double)(r1[k] - r0[k] + 1);
        f[3] = (double)(c1[k] - c0[k] + 1);
        f[4] = (double)r0[k] + (double)sr[k] / da;
        f[5] = (double)c0[k] + (double)sc[k] / da;
        const __int128 mrr = (__int128)a * srr[k] - (__int128)sr[k] * sr[k];
        const __int128 mcc = (__int128)a * scc[k] - (__int128)sc[k] * sc[k];
        const __int128 mrc = (__int128)a * src[k] - (__int128)sr[k] * sc[k];
        const double a2 = da * da;
        const double vrr = (double)mrr / a2, vcc = (double)mcc / a2, vrc = (double)mrc / a2;
        const double half = (vrr + vcc) / 2.0, dh = (vrr - vcc) / 2.0;
        const double disc = sqrt(dh * dh + vrc * vrc);
        const double l1 = half + disc;
        double l2 = half - disc;
        if (l2 < 0.0) l2 = 0.0;
        f[6] = 4.0 * sqrt(l1);
        f[7] = 4.0 * sqrt(l2);
        f[8] = l1 > 0.0 ? sqrt(1.0 - l2 / l1) : 0.0;
        const double P = (double)per[k];
        f[9] = 4.0 * 3.14159265358979323846 * da / (P * P);
        const int64_t *h = hist + k * 256;
        int64_t s1 = 0, s2 = 0, cum = 0;
        int vmin = -1, vmax = -1, med = -1;
        for (int v = 0; v < 256; v++) {
            if (!h[v]) continue;
            s1 += (int64_t)v * h[v];
            s2 += (int64_t)v * v * h[v];
            if (vmin < 0) vmin = v;
            vmax = v;
        }
        for (int v = 0; v < 256 && med < 0; v++) {
            cum += h[v];
            if (2 * cum >= a) med = v;
        }
        f[10] = (double)s1 / da;
        f[11] = sqrt((double)((__int128)a * s2 - (__int128)s1 * s1) / a2);
        f[12] = vmin;
        f[13] = vmax;
        f[14] = med;
        double ent = 0.0;
        for (int v = 0; v < 256; v++)
            if (h[v]) {
                const double p = (double)h[v] / da;
                ent -= p * log2(p);
            }
        f[15] = ent;
        const int64_t *g = glcm + k * 64;
        int64_t n2 = 0, con = 0, en = 0;
        for (int q = 0; q < 64; q++) {
            const int64_t d = (q >> 3) - (q & 7);
            n2 += g[q];
            con += d * d * g[q];
            en += g[q] * g[q];
        }
        f[16] = (double)n2;
        if (n2 > 0) {
            double hom = 0.0;
            for (int q = 0; q < 64; q++) {
                const int d = (q >> 3) - (q & 7);
                hom += (double)g[q] / (double)(1 + (d < 0 ? -d : d));
            }
            f[17] = (double)con / (double)n2;
            f[18] = (double)en / ((double)n2 * (double)n2);
            f[19] = hom / (double)n2;
        } else {
            f[17] = f[18] = f[19] = 0.0;
        }
    }
    free(lab); free(area); free(per); free(r0); free(c0); free(r1); free(c1); free(hist); free(glcm);
    free(sr); free(sc); free(srr); free(scc); free(src);
    return 0;
}

/* -------------------------------------------------------------- watershed */
/* Watershed after the Pre-Watershed step (Section 5.1), splitting touching
 * nuclei: marker-controlled flooding of the distance map D inside every
 * object of L (-1 outside; objects never exchange pixels). Pixels are
 * 8-connected within their object. For each object:
 *   1. markers: the regional maxima of the h-maxima transform
 *      R = reconstruction by dilation of max(D - h, 0) under D (within the
 *      object); a regional maximum is an 8-connected plateau of equal R with
 *      no neighbour of higher R; its label is the smallest linear index
 *      r * W + c of its pixels;
 *   2. flooding by levels (Vincent and Soille's geodesic influence zones):
 *      for every distinct value t of D in the object, from the highest down,
 *      the labelled pixels grow, in synchronous breadth-first layers, into
 *      the unlabelled pixels with D >= t; a pixel reached in a layer takes
 *      the smallest label among its labelled neighbours of the layers
 *      before (equally near basins: the smaller label).
 * B = the basin label of every object pixel, -1 elsewhere; *n_basins = the
 * number of markers. */
int orc_watershed(const int32_t *L, const int32_t *D, int H, int W, int h, int32_t *B, int *n_basins)
{
    if (!L || !D || !B || H < 1 || W < 1 || h < 0 || !n_basins) return -1;
    const long N = (long)H * W;
    int32_t *R = malloc(sizeof(int32_t) * (size_t)N);
    uint8_t *nm = malloc((size_t)N);
    long *queue = malloc(sizeof(long) * (size_t)N);
    long *next = malloc(sizeof(long) * (size_t)N);
    int32_t *cand = malloc(sizeof(int32_t) * (size_t)N);
    long *slot = malloc(sizeof(long) * (size_t)N);   /* a pixel's place in the next layer, or -1 */
    if (!R || !nm || !queue || !next || !cand || !slot) {
        free(R); free(nm); free(queue); free(next); free(cand); free(slot); free(slot);
        return -2;
    }
    for (long p = 0; p < N; p++) slot[p] = -1;
    static const int DR[8] = {-1, -1, -1, 0, 0, 1, 1, 1}, DC[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    /* 1a. h-maxima: R = max(D - h, 0) on object pixels, then raise every
     * pixel to min(D, max of R over itself and its object neighbours) in
     * forward and backward raster passes until a pass changes nothing */
    for (long p = 0; p < N; p++) R[p] = L[p] >= 0 ? (D[p] - h > 0 ? D[p] - h : 0) : 0;
    for (int changed = 1; changed;) {
        changed = 0;
        for (int dir = 0; dir < 2; dir++)
            for (long i = 0; i < N; i++) {
                const long p = dir ? N - 1 - i : i;
                if (L[p] < 0) continue;
                const int r = (int)(p / W), c = (int)(p % W);
                int32_t m = R[p];
                for (int e = 0; e < 8; e++) {
                    const int rr = r + DR[e], cc = c + DC[e];
                    if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                    const long q = (long)rr * W + cc;
                    if (L[q] == L[p] && R[q] > m) m = R[q];
                }
                if (m > D[p]) m = D[p];
                if (m > R[p]) {
                    R[p] = m;
                    changed = 1;
                }
            }
    }
    /* 1b. not a maximum: a higher neighbour, or an equal neighbour that is
     * not a maximum (spread over plateaus until nothing changes) */
    for (long p = 0; p < N; p++) {
        nm[p] = 0;
        if (L[p] < 0) continue;
        const int r = (int)(p / W), c = (int)(p % W);
        for (int e = 0; e < 8; e++) {
            const int rr = r + DR[e], cc = c + DC[e];
            if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
            const long q = (long)rr * W + cc;
            if (L[q] == L[p] && R[q] > R[p]) nm[p] = 1;
        }
    }
    for (int changed = 1; changed;) {
        changed = 0;
        for (long p = 0; p < N; p++) {
            if (L[p] < 0 || nm[p]) continue;
            const int r = (int)(p / W), c = (int)(p % W);
            for (int e = 0; e < 8; e++) {
                const int rr = r + DR[e], cc = c + DC[e];
                if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                const long q = (long)rr * W + cc;
                if (L[q] == L[p] && R[q] == R[p] && nm[q]) {
                    nm[p] = 1;
                    changed = 1;
                    break;
                }
            }
        }
    }
    /* 1c. marker labels: breadth-first over each plateau of maxima from its
     * first pixel in raster order (its smallest index) */
    for (long p = 0; p < N; p++) B[p] = -1;
    int nb = 0;
    for (long p = 0; p < N; p++) {
        if (L[p] < 0 || nm[p] || B[p] >= 0) continue;
        long head = 0, tail = 0;
        queue[tail++] = p;
        B[p] = (int32_t)p;
        nb++;
        while (head < tail) {
            const long x = queue[head++];
            const int r = (int)(x / W), c = (int)(x % W);
            for (int e = 0; e < 8; e++) {
                const int rr = r + DR[e], cc = c + DC[e];
                if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                const long q = (long)rr * W + cc;
                if (L[q] == L[p] && !nm[q] && B[q] < 0) {
                    B[q] = (int32_t)p;
                    queue[tail++] = q;
                }
            }
        }
    }
    *n_basins = nb;
    /* 2. flooding, one object at a time: its pixels in raster order */
    int32_t *lab = NULL;
    const long nobj = distinct_labels(L, N, &lab);
    if (nobj < 0) {
        free(R); free(nm); free(queue); free(next); free(cand); free(slot);
        return -2;
    }
    long *start = calloc((size_t)nobj + 1, sizeof(long));
    long *pix = malloc(sizeof(long) * (size_t)(N > 0 ? N : 1));
    int32_t *levels = malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
    if (!start || !pix || !levels) {
        free(R); free(nm); free(queue); free(next); free(cand); free(slot); free(lab); free(start); free(pix); free(levels);
        return -2;
    }
    for (long p = 0; p < N; p++)
        if (L[p] >= 0) start[find_sorted(lab, nobj, L[p]) + 1]++;
    for (long k = 0; k < nobj; k++) start[k + 1] += start[k];
    {
        long *fill = calloc((size_t)nobj + 1, sizeof(long));
        if (!fill) {
            free(R); free(nm); free(queue); free(next); free(cand); free(slot); free(lab); free(start); free(pix); free(levels);
            return -2;
        }
        for (long p = 0; p < N; p++)
            if (L[p] >= 0) {
                const long k = find_sorted(lab, nobj, L[p]);
                pix[start[k] + fill[k]++] = p;
            }
        free(fill);
    }
    for (long k = 0; k < nobj; k++) {
        const long a = start[k], b = start[k + 1];
        long nl = 0;
        for (long i = a; i < b; i++) levels[nl++] = D[pix[i]];
        qsort(levels, (size_t)nl, sizeof(int32_t), cmp_i32);
        for (long li = nl - 1; li >= 0; li--) {
            if (li < nl - 1 && levels[li] == levels[li + 1]) continue;
            const int32_t t = levels[li];
            /* layer 0: every labelled pixel of the object */
            long nf = 0;
            for (long i = a; i < b; i++)
                if (B[pix[i]] >= 0) queue[nf++] = pix[i];
            for (;;) {
                /* the next layer: unlabelled pixels with D >= t next to the
                 * current layer, each with the smallest label among those
                 * neighbours (collected first, assigned after) */
                long nn = 0;
                for (long f = 0; f < nf; f++) {
                    const long x = queue[f];
                    const int r = (int)(x / W), c = (int)(x % W);
                    for (int e = 0; e < 8; e++) {
                        const int rr = r + DR[e], cc = c + DC[e];
                        if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                        const long q = (long)rr * W + cc;
                        if (L[q] != L[x] || B[q] >= 0 || D[q] < t) continue;
                        if (slot[q] < 0) {
                            slot[q] = nn;
                            next[nn] = q;
                            cand[nn] = B[x];
                            nn++;
                        } else if (B[x] < cand[slot[q]]) {
                            cand[slot[q]] = B[x];
                        }
                    }
                }
                if (nn == 0) break;
                for (long j = 0; j < nn; j++) {
                    B[next[j]] = cand[j];
                    slot[next[j]] = -1;
                }
                for (long j = 0; j < nn; j++) queue[j] = next[j];
                nf = nn;
            }
        }
    }
    free(R); free(nm); free(queue); free(next); free(cand); free(slot); free(lab); free(start); free(pix); free(levels);
    return 0;
}
