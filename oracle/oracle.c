/*
 * CPU ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously correct CPU implementations of the segmentation ops
 * that the paper runs as fine-grain GPU tasks (Teodoro et al., "Region
 * Templates", Section 5.1 "Example Application": ReconToNuclei, FillHoles,
 * Pre-Watershed, BWLabel; Section 3.2.1 "PATS": AreaThreshold, FillHoles).
 * The paper names these operations and defers their definitions to earlier
 * work, so every function below follows the textbook definition it cites.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library. The GPU product path never calls it, and
 * this file shares no code with the CUDA sources.
 *
 * Conventions: images are row-major and contiguous (row stride = W), pixel
 * p = r*W + c. Out-of-image neighbours do not exist. conn is 4 or 8.
 * Binary inputs: any nonzero byte is foreground. Return value 0 = ok,
 * -1 = bad argument, -2 = out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const int DR8[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
static const int DC8[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
static const int DR4[4] = {-1, 0, 0, 1};
static const int DC4[4] = {0, -1, 1, 0};

static int nbr_count(int conn) { return conn == 8 ? 8 : 4; }
static int nbr_dr(int conn, int k) { return conn == 8 ? DR8[k] : DR4[k]; }
static int nbr_dc(int conn, int k) { return conn == 8 ? DC8[k] : DC4[k]; }

/* ------------------------------------------------------------------ marker */
/* Marker of the ReconToNuclei step for the nuclei tiles: J = max(I - h, 0)
 * inside the tile, and J = I on the one-pixel border (all four edges). */
void orc_marker(const uint8_t *I, int H, int W, int h, uint8_t *J)
{
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            long p = (long)r * W + c;
            int v = (int)I[p] - h;
            if (r == 0 || c == 0 || r == H - 1 || c == W - 1)
                J[p] = I[p];
            else
                J[p] = (uint8_t)(v > 0 ? v : 0);
        }
}

/* ------------------------------------------------ reconstruction by dilation */
/* ReconToNuclei (Section 5.1) is grayscale morphological reconstruction by
 * dilation of marker J under mask I. Definition (Vincent 1993, "Morphological
 * grayscale reconstruction in image analysis", IEEE TIP 2(2)): the limit of
 * repeated elementary geodesic dilations
 *     R_0 = min(J, I),   R_{k+1} = min(delta(R_k), I),
 * where delta takes the maximum over the pixel and its conn-neighbours, run
 * until R_{k+1} = R_k. A marker above the mask is clamped by R_0 = min(J, I).
 * Each step is computed from the previous image only (Jacobi order), exactly
 * as the definition reads. *iters receives the number of steps that changed
 * something. */
int orc_recon_fixpoint(const uint8_t *J, const uint8_t *I, int H, int W, int conn,
                       uint8_t *R, long *iters)
{
    if (H < 1 || W < 1 || (conn != 4 && conn != 8)) return -1;
    long N = (long)H * W;
    uint8_t *prev = (uint8_t *)malloc((size_t)N);
    if (!prev) return -2;
    for (long p = 0; p < N; p++) R[p] = J[p] < I[p] ? J[p] : I[p];
    long k = 0;
    for (;;) {
        memcpy(prev, R, (size_t)N);
        int changed = 0;
        for (int r = 0; r < H; r++)
            for (int c = 0; c < W; c++) {
                long p = (long)r * W + c;
                int m = prev[p];
                for (int n = 0; n < nbr_count(conn); n++) {
                    int rr = r + nbr_dr(conn, n), cc = c + nbr_dc(conn, n);
                    if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                    int v = prev[(long)rr * W + cc];
                    if (v > m) m = v;
                }
                if (m > I[p]) m = I[p];
                if (m != R[p]) { R[p] = (uint8_t)m; changed = 1; }
            }
        if (!changed) break;
        k++;
    }
    if (iters) *iters = k;
    free(prev);
    return 0;
}

/* Vincent's hybrid reconstruction algorithm (Vincent 1993, Section V): one
 * raster scan and one anti-raster scan that propagate through the causal
 * half-neighbourhoods, followed by a FIFO propagation seeded by the pixels
 * the anti-raster scan leaves able to raise a neighbour. It reaches the same
 * fixed point as orc_recon_fixpoint and is fast enough for 4K x 4K tiles. */
int orc_recon_vincent(const uint8_t *J, const uint8_t *I, int H, int W, int conn, uint8_t *R)
{
    if (H < 1 || W < 1 || (conn != 4 && conn != 8)) return -1;
    long N = (long)H * W;
    long *fifo = (long *)malloc(sizeof(long) * (size_t)(N + 1));
    if (!fifo) return -2;
    long head = 0, tail = 0;   /* ring buffer of capacity N + 1 */
    for (long p = 0; p < N; p++) R[p] = J[p] < I[p] ? J[p] : I[p];

    /* raster scan: N+ = already-visited neighbours (row above, left) */
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            long p = (long)r * W + c;
            int m = R[p];
            for (int n = 0; n < nbr_count(conn); n++) {
                int dr = nbr_dr(conn, n), dc = nbr_dc(conn, n);
                if (!(dr < 0 || (dr == 0 && dc < 0))) continue;
                int rr = r + dr, cc = c + dc;
                if (rr < 0 || cc < 0 || cc >= W) continue;
                int v = R[(long)rr * W + cc];
                if (v > m) m = v;
            }
            R[p] = (uint8_t)(m < I[p] ? m : I[p]);
        }

    /* anti-raster scan: N- = neighbours after p in raster order */
    for (int r = H - 1; r >= 0; r--)
        for (int c = W - 1; c >= 0; c--) {
            long p = (long)r * W + c;
            int m = R[p];
            for (int n = 0; n < nbr_count(conn); n++) {
                int dr = nbr_dr(conn, n), dc = nbr_dc(conn, n);
                if (!(dr > 0 || (dr == 0 && dc > 0))) continue;
                int rr = r + dr, cc = c + dc;
                if (rr >= H || cc < 0 || cc >= W) continue;
                int v = R[(long)rr * W + cc];
                if (v > m) m = v;
            }
            R[p] = (uint8_t)(m < I[p] ? m : I[p]);
            for (int n = 0; n < nbr_count(conn); n++) {
                int dr = nbr_dr(conn, n), dc = nbr_dc(conn, n);
                if (!(dr > 0 || (dr == 0 && dc > 0))) continue;
                int rr = r + dr, cc = c + dc;
                if (rr >= H || cc < 0 || cc >= W) continue;
                long q = (long)rr * W + cc;
                if (R[q] < R[p] && R[q] < I[q]) {
                    fifo[tail] = p;
                    tail = (tail + 1) % (N + 1);
                    break;
                }
            }
        }

    /* FIFO propagation */
    while (head != tail) {
        long p = fifo[head];
        head = (head + 1) % (N + 1);
        int r = (int)(p / W), c = (int)(p % W);
        for (int n = 0; n < nbr_count(conn); n++) {
            int rr = r + nbr_dr(conn, n), cc = c + nbr_dc(conn, n);
            if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
            long q = (long)rr * W + cc;
            if (R[q] < R[p] && I[q] != R[q]) {
                R[q] = R[p] < I[q] ? R[p] : I[q];
                fifo[tail] = q;
                tail = (tail + 1) % (N + 1);
            }
        }
    }
    free(fifo);
    return 0;
}

/* ----------------------------------------------------------------- threshold */
/* Binarisation ahead of FillHoles: B = 1 where R < t (dark nuclei). */
void orc_threshold_below(const uint8_t *R, long N, int t, uint8_t *B)
{
    for (long p = 0; p < N; p++) B[p] = (uint8_t)(R[p] < t ? 1 : 0);
}

/* ---------------------------------------------------------------- fill holes */
/* FillHoles (Sections 3.2.1, 5.1): a hole is a background region that no
 * conn-path of background pixels links to the tile border. The output is 1 on
 * the foreground and on every hole, 0 on background reachable from the
 * border. Computed by breadth-first search over background pixels, seeded
 * with every background pixel on the border. */
int orc_fill_holes(const uint8_t *B, int H, int W, int conn, uint8_t *F)
{
    if (H < 1 || W < 1 || (conn != 4 && conn != 8)) return -1;
    long N = (long)H * W;
    long *queue = (long *)malloc(sizeof(long) * (size_t)N);
    uint8_t *reached = (uint8_t *)calloc((size_t)N, 1);
    if (!queue || !reached) { free(queue); free(reached); return -2; }
    long head = 0, tail = 0;
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            long p = (long)r * W + c;
            int on_border = (r == 0 || c == 0 || r == H - 1 || c == W - 1);
            if (on_border && B[p] == 0 && !reached[p]) { reached[p] = 1; queue[tail++] = p; }
        }
    while (head < tail) {
        long p = queue[head++];
        int r = (int)(p / W), c = (int)(p % W);
        for (int n = 0; n < nbr_count(conn); n++) {
            int rr = r + nbr_dr(conn, n), cc = c + nbr_dc(conn, n);
            if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
            long q = (long)rr * W + cc;
            if (B[q] == 0 && !reached[q]) { reached[q] = 1; queue[tail++] = q; }
        }
    }
    for (long p = 0; p < N; p++) F[p] = (uint8_t)((B[p] != 0 || !reached[p]) ? 1 : 0);
    free(queue);
    free(reached);
    return 0;
}

/* ------------------------------------------------- labeling and area filter */
/* BWLabel (Section 5.1) labels the conn-connected components of the
 * foreground; AreaThreshold (Section 3.2.1) drops components whose area lies
 * outside [min_area, max_area] (both ends kept). The label of a component is
 * the smallest linear index r*W + c of its pixels; background and dropped
 * pixels get -1. Components are found by breadth-first search started from
 * pixels in raster order, so the start pixel is the component's smallest
 * index. *n_kept receives the number of components kept. */
int orc_label_area(const uint8_t *F, int H, int W, int conn, int min_area, int max_area,
                   int32_t *L, int32_t *n_kept)
{
    if (H < 1 || W < 1 || (conn != 4 && conn != 8)) return -1;
    long N = (long)H * W;
    long *queue = (long *)malloc(sizeof(long) * (size_t)N);
    if (!queue) return -2;
    for (long p = 0; p < N; p++) L[p] = -1;
    int32_t kept = 0;
    for (long s = 0; s < N; s++) {
        if (F[s] == 0 || L[s] != -1) continue;
        long head = 0, tail = 0;
        L[s] = (int32_t)s;
        queue[tail++] = s;
        while (head < tail) {
            long p = queue[head++];
            int r = (int)(p / W), c = (int)(p % W);
            for (int n = 0; n < nbr_count(conn); n++) {
                int rr = r + nbr_dr(conn, n), cc = c + nbr_dc(conn, n);
                if (rr < 0 || rr >= H || cc < 0 || cc >= W) continue;
                long q = (long)rr * W + cc;
                if (F[q] != 0 && L[q] == -1) { L[q] = (int32_t)s; queue[tail++] = q; }
            }
        }
        /* queue[0..tail) holds exactly this component: its area is tail */
        if (tail < min_area || tail > max_area) {
            for (long i = 0; i < tail; i++) L[queue[i]] = -2;   /* dropped, fixed below */
        } else {
            kept++;
        }
    }
    for (long p = 0; p < N; p++) if (L[p] == -2) L[p] = -1;
    if (n_kept) *n_kept = kept;
    free(queue);
    return 0;
}

/* ----------------------------------------------------- distance transform */
/* Exact squared Euclidean distance transform, the input of the
 * Pre-Watershed step (Section 5.1): for every pixel p,
 *     D(p) = min over background pixels q of (r_p - r_q)^2 + (c_p - c_q)^2,
 * with background = fg == 0 and only in-image pixels counting. D = 0 on the
 * background. If the image has no background pixel at all, D = -1 everywhere.
 * Brute force: every pixel against every background pixel. */
int orc_edt_brute(const uint8_t *fg, int H, int W, int32_t *D)
{
    if (H < 1 || W < 1) return -1;
    long N = (long)H * W;
    for (long p = 0; p < N; p++) {
        int r = (int)(p / W), c = (int)(p % W);
        int64_t best = -1;
        for (long q = 0; q < N; q++) {
            if (fg[q] != 0) continue;
            int64_t dr = r - (int)(q / W), dc = c - (int)(q % W);
            int64_t d = dr * dr + dc * dc;
            if (best < 0 || d < best) best = d;
        }
        D[p] = (int32_t)best;
    }
    return 0;
}

/* The same definition evaluated at one pixel (for sampled checks on images
 * too large for the brute force over every pixel). */
int64_t orc_edt_at(const uint8_t *fg, int H, int W, int r, int c)
{
    int64_t best = -1;
    for (int rr = 0; rr < H; rr++)
        for (int cc = 0; cc < W; cc++) {
            if (fg[(long)rr * W + cc] != 0) continue;
            int64_t dr = r - rr, dc = c - cc;
            int64_t d = dr * dr + dc * dc;
            if (best < 0 || d < best) best = d;
        }
    return best;
}

/* Meijster, Roerdink, Hesselink 2000 ("A general algorithm for computing
 * distance transforms in linear time"), Euclidean case, 64-bit integers.
 * Phase 1: per column, g = vertical distance to the nearest background pixel
 * in that column (INF when the column has none), by a downward and an upward
 * scan. Phase 2: per row, the lower envelope of the parabolas
 * f_u(x) = (x - u)^2 + g(u)^2, built left to right with the separator
 * Sep(i, u) = floor((u^2 - i^2 + g(u)^2 - g(i)^2) / (2 (u - i))), then read
 * back right to left. INF = H + W exceeds every real distance, so a parabola
 * of an empty column never wins when some background exists. */
int orc_edt_meijster(const uint8_t *fg, int H, int W, int32_t *D)
{
    if (H < 1 || W < 1) return -1;
    long N = (long)H * W;
    int64_t INF = (int64_t)H + W;
    int64_t *g = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *s = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    int64_t *t = (int64_t *)malloc(sizeof(int64_t) * (size_t)W);
    if (!g || !s || !t) { free(g); free(s); free(t); return -2; }
    int any_bg = 0;
    for (long p = 0; p < N; p++) if (fg[p] == 0) { any_bg = 1; break; }
    if (!any_bg) {
        for (long p = 0; p < N; p++) D[p] = -1;
        free(g); free(s); free(t);
        return 0;
    }
    for (int x = 0; x < W; x++) {
        g[x] = fg[x] == 0 ? 0 : INF;
        for (int y = 1; y < H; y++) {
            long p = (long)y * W + x;
            g[p] = fg[p] == 0 ? 0 : (g[p - W] >= INF ? INF : g[p - W] + 1);
        }
        for (int y = H - 2; y >= 0; y--) {
            long p = (long)y * W + x;
            if (g[p + W] + 1 < g[p]) g[p] = g[p + W] + 1;
        }
    }
    for (int y = 0; y < H; y++) {
        const int64_t *gy = g + (long)y * W;
        long q = 0;
        s[0] = 0;
        t[0] = 0;
        for (int u = 1; u < W; u++) {
            /* f_i(t_q) > f_u(t_q): u hides the last segment */
            while (q >= 0) {
                int64_t i = s[q], x = t[q];
                int64_t fi = (x - i) * (x - i) + gy[i] * gy[i];
                int64_t fu = (x - u) * (x - u) + gy[u] * gy[u];
                if (fi > fu) q--; else break;
            }
            if (q < 0) {
                q = 0;
                s[0] = u;
            } else {
                int64_t i = s[q];
                int64_t num = (int64_t)u * u - i * i + gy[u] * gy[u] - gy[i] * gy[i];
                int64_t den = 2 * ((int64_t)u - i);
                int64_t w = num / den;              /* num >= 0 here would floor; */
                if ((num % den != 0) && ((num < 0) != (den < 0))) w--;   /* floor */
                w += 1;
                if (w < W) {
                    q++;
                    s[q] = u;
                    t[q] = w;
                }
            }
        }
        for (int u = W - 1; u >= 0; u--) {
            int64_t i = s[q];
            int64_t d = ((int64_t)u - i) * ((int64_t)u - i) + gy[i] * gy[i];
            D[(long)y * W + u] = (int32_t)d;
            if (u == t[q]) q--;
        }
    }
    free(g); free(s); free(t);
    return 0;
}

/* ------------------------------------------------------------------ chain */
/* The segmentation chain of the nuclei tiles, in this order:
 *   J = marker(I, h); R = recon(J, I, conn_recon); B = (R < t);
 *   F = fill_holes(B, conn_fill); L = label_area(F, 8, [amin, amax]);
 *   D = edt(L >= 0).
 * Any of R, F may be NULL (then scratch is used). Reconstruction uses
 * Vincent's algorithm. Returns 0 on success. */
int orc_chain(const uint8_t *I, int H, int W, int h, int conn_recon, int t, int conn_fill,
              int amin, int amax, uint8_t *R_out, uint8_t *F_out, int32_t *L, int32_t *D,
              int32_t *n_kept)
{
    if (H < 1 || W < 1) return -1;
    long N = (long)H * W;
    uint8_t *J = (uint8_t *)malloc((size_t)N);
    uint8_t *R = R_out ? R_out : (uint8_t *)malloc((size_t)N);
    uint8_t *B = (uint8_t *)malloc((size_t)N);
    uint8_t *F = F_out ? F_out : (uint8_t *)malloc((size_t)N);
    uint8_t *fg = (uint8_t *)malloc((size_t)N);
    int rc = -2;
    if (!J || !R || !B || !F || !fg) goto done;
    orc_marker(I, H, W, h, J);
    if ((rc = orc_recon_vincent(J, I, H, W, conn_recon, R)) != 0) goto done;
    orc_threshold_below(R, N, t, B);
    if ((rc = orc_fill_holes(B, H, W, conn_fill, F)) != 0) goto done;
    if ((rc = orc_label_area(F, H, W, 8, amin, amax, L, n_kept)) != 0) goto done;
    for (long p = 0; p < N; p++) fg[p] = (uint8_t)(L[p] >= 0 ? 1 : 0);
    rc = orc_edt_meijster(fg, H, W, D);
done:
    free(J);
    if (!R_out) free(R);
    free(B);
    if (!F_out) free(F);
    free(fg);
    return rc;
}
