/*
 * ec_oracle.c -- plain, slow, single-threaded CPU oracle (see ec_oracle.h).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  Written from the
 * thesis text (Eilemann, arXiv 1902.08755), chapter 5 "Compositing"; it shares
 * no code with the CUDA library.  Each routine is the plain definition of what
 * it computes, pixel by pixel, with no blocking, fusion or reordering.
 */
#include "ec_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ rects */

static int rect_valid(orc_rect r) { return r.w >= 0 && r.h >= 0; }

static int rect_empty(orc_rect r) { return r.w <= 0 || r.h <= 0; }

static int rect_inside(orc_rect inner, orc_rect outer)
{
    if (rect_empty(inner)) return 1;
    return inner.x >= outer.x && inner.y >= outer.y &&
           (int64_t)inner.x + inner.w <= (int64_t)outer.x + outer.w &&
           (int64_t)inner.y + inner.h <= (int64_t)outer.y + outer.h;
}

static int rect_contains(orc_rect r, int32_t px, int32_t py)
{
    return px >= r.x && py >= r.y && (int64_t)px < (int64_t)r.x + r.w &&
           (int64_t)py < (int64_t)r.y + r.h;
}

static orc_rect rect_intersect(orc_rect a, orc_rect b)
{
    int64_t x0 = a.x > b.x ? a.x : b.x;
    int64_t y0 = a.y > b.y ? a.y : b.y;
    int64_t x1 = (int64_t)a.x + a.w < (int64_t)b.x + b.w ? (int64_t)a.x + a.w : (int64_t)b.x + b.w;
    int64_t y1 = (int64_t)a.y + a.h < (int64_t)b.y + b.h ? (int64_t)a.y + a.h : (int64_t)b.y + b.h;
    orc_rect r = {0, 0, 0, 0};
    if (x1 > x0 && y1 > y0) {
        r.x = (int32_t)x0; r.y = (int32_t)y0;
        r.w = (int32_t)(x1 - x0); r.h = (int32_t)(y1 - y0);
    }
    return r;
}

/* Thesis 5.3: the ROI of a composited frame is combined with the ROIs of its
 * inputs for the next readback.  Here the combination is the bounding box of
 * the union of the sources' ROIs, clipped to the output viewport. */
static orc_rect merge_rois(const orc_rect* roi, int32_t n, orc_rect out_pvp)
{
    orc_rect acc = {0, 0, 0, 0};
    int have = 0;
    int64_t x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    for (int32_t i = 0; i < n; ++i) {
        orc_rect c = rect_intersect(roi[i], out_pvp);
        if (rect_empty(c)) continue;
        if (!have) {
            x0 = c.x; y0 = c.y; x1 = (int64_t)c.x + c.w; y1 = (int64_t)c.y + c.h;
            have = 1;
        } else {
            if (c.x < x0) x0 = c.x;
            if (c.y < y0) y0 = c.y;
            if ((int64_t)c.x + c.w > x1) x1 = (int64_t)c.x + c.w;
            if ((int64_t)c.y + c.h > y1) y1 = (int64_t)c.y + c.h;
        }
    }
    if (have) {
        acc.x = (int32_t)x0; acc.y = (int32_t)y0;
        acc.w = (int32_t)(x1 - x0); acc.h = (int32_t)(y1 - y0);
    }
    return acc;
}

static int check_image(orc_rect pvp, orc_rect roi, int32_t pitch)
{
    if (!rect_valid(pvp) || !rect_valid(roi)) return 0;
    if (pitch < pvp.w) return 0;
    if (!rect_inside(roi, pvp)) return 0;
    return 1;
}

/* --------------------------------------------------- depth compositing --- */

/* Thesis 5.2.1: in depth-sorted compositing each output pixel takes the colour
 * of the source whose depth value is nearest the viewer.  Thesis 3.6: inputs
 * are merged in whatever order they arrive, so the result may not depend on
 * order; ties therefore go to the lower source index, which makes the merge a
 * lexicographic minimum over (depth, i). */
int orc_composite_depth(const orc_depth_src* src, int32_t n, int32_t color_bytes,
                        orc_rect out_pvp, int32_t out_pitch, void* out_color,
                        float* out_depth, int16_t* winner, orc_rect* out_roi)
{
    if (n < 0 || !rect_valid(out_pvp) || out_pitch < out_pvp.w) return ORC_EINVAL;
    if (color_bytes != 4 && color_bytes != 8 && color_bytes != 16) return ORC_EINVAL;
    if (n > 0 && !src) return ORC_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (!check_image(src[i].pvp, src[i].roi, src[i].pitch)) return ORC_EINVAL;

    const size_t npx = (size_t)out_pvp.w * (size_t)out_pvp.h;
    float* best_d = (float*)malloc((npx ? npx : 1) * sizeof(float));
    int32_t* best_i = (int32_t*)malloc((npx ? npx : 1) * sizeof(int32_t));
    if (!best_d || !best_i) { free(best_d); free(best_i); return ORC_EINVAL; }

    /* cleared destination: depth 1.0, no source */
    for (size_t p = 0; p < npx; ++p) { best_d[p] = 1.0f; best_i[p] = -1; }

    for (int32_t i = 0; i < n; ++i) {
        orc_rect a = rect_intersect(src[i].roi, out_pvp);
        for (int32_t py = a.y; py < a.y + a.h; ++py) {
            for (int32_t px = a.x; px < a.x + a.w; ++px) {
                size_t e = (size_t)(py - src[i].pvp.y) * (size_t)src[i].pitch +
                           (size_t)(px - src[i].pvp.x);
                size_t p = (size_t)(py - out_pvp.y) * (size_t)out_pvp.w + (size_t)(px - out_pvp.x);
                float d = src[i].depth[e];
                if (d < best_d[p]) { best_d[p] = d; best_i[p] = i; }
            }
        }
    }

    for (int32_t py = 0; py < out_pvp.h; ++py) {
        for (int32_t px = 0; px < out_pvp.w; ++px) {
            size_t p = (size_t)py * out_pvp.w + px;
            size_t o = (size_t)py * out_pitch + px;
            unsigned char* dst = (unsigned char*)out_color + o * color_bytes;
            int32_t i = best_i[p];
            if (i < 0) {
                memset(dst, 0, (size_t)color_bytes);
            } else {
                size_t e = (size_t)(py + out_pvp.y - src[i].pvp.y) * (size_t)src[i].pitch +
                           (size_t)(px + out_pvp.x - src[i].pvp.x);
                memcpy(dst, (const unsigned char*)src[i].color + e * color_bytes, (size_t)color_bytes);
            }
            if (out_depth) out_depth[o] = best_d[p];
            if (winner) winner[p] = (int16_t)i;
        }
    }
    if (out_roi) {
        orc_rect* r = (orc_rect*)malloc((n ? n : 1) * sizeof(orc_rect));
        for (int32_t i = 0; i < n; ++i) r[i] = src[i].roi;
        *out_roi = merge_rois(r, n, out_pvp);
        free(r);
    }
    free(best_d);
    free(best_i);
    return ORC_OK;
}

/* ------------------------------------------------ alpha (over) compositing */

/* IEEE-754 binary16 to double, exactly: value = (-1)^s * m * 2^(e-25) with the
 * implicit leading one for normal numbers. */
static double half_to_double(uint16_t h)
{
    int s = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int m = h & 0x3ff;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m + 1024), e - 25);
    return s ? -v : v;
}

static void load_rgba(const orc_layer* l, int32_t fmt, int32_t px, int32_t py, double c[4])
{
    size_t e = (size_t)(py - l->pvp.y) * (size_t)l->pitch + (size_t)(px - l->pvp.x);
    if (fmt == ORC_F32) {
        const float* f = (const float*)l->color + 4 * e;
        for (int k = 0; k < 4; ++k) c[k] = (double)f[k];
    } else {
        const uint16_t* h = (const uint16_t*)l->color + 4 * e;
        for (int k = 0; k < 4; ++k) c[k] = half_to_double(h[k]);
    }
}

static int check_layers(const orc_layer* layers, int32_t n, int32_t fmt, const int32_t* order)
{
    if (n < 0 || (n > 0 && !layers)) return 0;
    if (fmt != ORC_F32 && fmt != ORC_F16) return 0;
    for (int32_t i = 0; i < n; ++i)
        if (!check_image(layers[i].pvp, layers[i].roi, layers[i].pitch)) return 0;
    if (order) {
        char* seen = (char*)calloc((size_t)(n ? n : 1), 1);
        for (int32_t k = 0; k < n; ++k) {
            if (order[k] < 0 || order[k] >= n || seen[order[k]]) { free(seen); return 0; }
            seen[order[k]] = 1;
        }
        free(seen);
    }
    return 1;
}

/* Thesis 5.2.1: the partial images of a spatial decomposition are blended in
 * their sorted order, which keeps transparency correct.  The blend is the
 * Porter-Duff "over" operator on premultiplied RGBA, front to back:
 *   C_0 = 0, T_0 = 1;  C_{k+1} = C_k + T_k c_k;  T_{k+1} = T_k (1 - a_k). */
int orc_composite_alpha(const orc_layer* layers, int32_t n, int32_t fmt,
                        const int32_t* order, orc_rect out_pvp, double* out,
                        double* t_final, orc_rect* out_roi)
{
    if (!rect_valid(out_pvp) || !check_layers(layers, n, fmt, order)) return ORC_EINVAL;
    for (int32_t py = out_pvp.y; py < out_pvp.y + out_pvp.h; ++py) {
        for (int32_t px = out_pvp.x; px < out_pvp.x + out_pvp.w; ++px) {
            double C[4] = {0.0, 0.0, 0.0, 0.0};
            double T = 1.0;
            for (int32_t k = 0; k < n; ++k) {
                const orc_layer* l = &layers[order ? order[k] : k];
                if (!rect_contains(l->roi, px, py)) continue; /* transparent */
                double c[4];
                load_rgba(l, fmt, px, py, c);
                for (int ch = 0; ch < 4; ++ch) C[ch] += T * c[ch];
                T *= 1.0 - c[3];
            }
            size_t p = (size_t)(py - out_pvp.y) * out_pvp.w + (size_t)(px - out_pvp.x);
            for (int ch = 0; ch < 4; ++ch) out[4 * p + ch] = C[ch];
            if (t_final) t_final[p] = T;
        }
    }
    if (out_roi) {
        orc_rect* r = (orc_rect*)malloc((n ? n : 1) * sizeof(orc_rect));
        for (int32_t i = 0; i < n; ++i) r[i] = layers[i].roi;
        *out_roi = merge_rois(r, n, out_pvp);
        free(r);
    }
    return ORC_OK;
}

/* Reverse-mode derivative of the front-to-back recurrence above for
 * L = sum_p sum_ch g[p][ch] out[p][ch]:
 *   out = sum_k T_k c_k,   T_k = prod_{m<k} (1 - a_m)
 *   dL/dc_k^{RGB} = g^{RGB} T_k
 *   dL/da_k       = g^A T_k - sum_{j>k} (g.c_j) T_j / (1 - a_k)
 *                 = T_k (g^A - R_k),  R_k = sum_{j>k} (g.c_j) prod_{k<m<j} (1 - a_m)
 * with R evaluated back to front: R_{n-1} = 0, R_{k-1} = g.c_k + (1 - a_k) R_k.
 * The premultiplied colour is an independent input (no chain rule through a
 * premultiplication the caller may have done). */
int orc_composite_alpha_backward(const orc_layer* layers, int32_t n, int32_t fmt,
                                 const int32_t* order, orc_rect out_pvp,
                                 const double* g, double* const* grad)
{
    if (!rect_valid(out_pvp) || !check_layers(layers, n, fmt, order)) return ORC_EINVAL;
    if (n > 0 && (!g || !grad)) return ORC_EINVAL;
    double* T = (double*)malloc(((size_t)n + 1) * sizeof(double));
    double* c = (double*)malloc(((size_t)n + 1) * 4 * sizeof(double));
    char* in = (char*)malloc((size_t)n + 1);
    for (int32_t py = out_pvp.y; py < out_pvp.y + out_pvp.h; ++py) {
        for (int32_t px = out_pvp.x; px < out_pvp.x + out_pvp.w; ++px) {
            size_t p = (size_t)(py - out_pvp.y) * out_pvp.w + (size_t)(px - out_pvp.x);
            const double* gp = g + 4 * p;
            /* forward: transmittance in front of every layer */
            T[0] = 1.0;
            for (int32_t k = 0; k < n; ++k) {
                const orc_layer* l = &layers[order ? order[k] : k];
                in[k] = (char)rect_contains(l->roi, px, py);
                if (in[k]) load_rgba(l, fmt, px, py, c + 4 * k);
                else for (int ch = 0; ch < 4; ++ch) c[4 * k + ch] = 0.0;
                T[k + 1] = T[k] * (1.0 - c[4 * k + 3]);
            }
            /* backward: R_k from the back */
            double R = 0.0;
            for (int32_t k = n - 1; k >= 0; --k) {
                int32_t i = order ? order[k] : k;
                const orc_layer* l = &layers[i];
                if (rect_contains(l->pvp, px, py)) {
                    size_t e = (size_t)(py - l->pvp.y) * (size_t)l->pitch + (size_t)(px - l->pvp.x);
                    double* d = grad[i] + 4 * e;
                    if (in[k]) {
                        d[0] = gp[0] * T[k];
                        d[1] = gp[1] * T[k];
                        d[2] = gp[2] * T[k];
                        d[3] = T[k] * (gp[3] - R);
                    } else {
                        d[0] = d[1] = d[2] = d[3] = 0.0;
                    }
                }
                const double* ck = c + 4 * k;
                double gc = gp[0] * ck[0] + gp[1] * ck[1] + gp[2] * ck[2] + gp[3] * ck[3];
                R = gc + (1.0 - ck[3]) * R;
            }
        }
    }
    free(T);
    free(c);
    free(in);
    return ORC_OK;
}

int orc_composite_depth_backward(const int16_t* winner, orc_rect out_pvp,
                                 const float* g, int32_t n, const orc_rect* pvps,
                                 const int32_t* pitches, float* const* grad)
{
    if (!rect_valid(out_pvp) || n < 0) return ORC_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (!rect_valid(pvps[i]) || pitches[i] < pvps[i].w) return ORC_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        orc_rect a = rect_intersect(pvps[i], out_pvp);
        for (int32_t py = a.y; py < a.y + a.h; ++py) {
            for (int32_t px = a.x; px < a.x + a.w; ++px) {
                size_t p = (size_t)(py - out_pvp.y) * out_pvp.w + (size_t)(px - out_pvp.x);
                size_t e = (size_t)(py - pvps[i].y) * (size_t)pitches[i] + (size_t)(px - pvps[i].x);
                float* d = grad[i] + 4 * e;
                for (int ch = 0; ch < 4; ++ch) d[ch] = winner[p] == i ? g[4 * p + ch] : 0.0f;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------ RLE codec --- */

#define ORC_MAGIC 0x31524345u /* "ECR1" little-endian */
#define ORC_VERSION 1u
#define ORC_CHUNK 4096u
#define ORC_HEADER 32u
#define ORC_MAX_ELEMS (1u << 28)

/* Thesis 5.5.1, swizzle preconditioner: reorder and interleave the component
 * bits by significance, so that the most significant bits of all components
 * end up together in one byte stream.  Component j (byte j of the element,
 * R,G,B,A = 0..3) is cut into four 2-bit groups, most significant first; output
 * byte k gathers group k of every component, component 0 in its top bits:
 *   s_k = sum_j ((b_j >> (6 - 2k)) & 3) << (6 - 2j).                          */
uint32_t orc_swizzle(uint32_t v)
{
    uint32_t out = 0;
    for (int k = 0; k < 4; ++k) {
        uint32_t s = 0;
        for (int j = 0; j < 4; ++j) {
            uint32_t b = (v >> (8 * j)) & 0xffu;
            s |= ((b >> (6 - 2 * k)) & 3u) << (6 - 2 * j);
        }
        out |= s << (8 * k);
    }
    return out;
}

/* Inverse of orc_swizzle, written as the inverse scatter of the definition:
 * bits (6-2j) of output byte k go back to group k of component j. */
uint32_t orc_unswizzle(uint32_t v)
{
    uint32_t out = 0;
    for (int k = 0; k < 4; ++k) {
        uint32_t s = (v >> (8 * k)) & 0xffu;
        for (int j = 0; j < 4; ++j) {
            uint32_t grp = (s >> (6 - 2 * j)) & 3u;
            out |= (grp << (6 - 2 * k)) << (8 * j);
        }
    }
    return out;
}

static uint64_t n_chunks_of(uint64_t n) { return (n + ORC_CHUNK - 1) / ORC_CHUNK; }

size_t orc_rle_max_size(int32_t w, int32_t h)
{
    if (w < 0 || h < 0) return 0;
    uint64_t n = (uint64_t)w * (uint64_t)h;
    uint64_t nc = n_chunks_of(n);
    uint64_t size = ORC_HEADER + 16u * nc;
    for (uint64_t c = 0; c < nc; ++c) {
        uint64_t len = (c + 1 < nc) ? ORC_CHUNK : n - c * ORC_CHUNK;
        size += 4u * (len + (len + 127) / 128);
    }
    return (size_t)size;
}

static void put_u32(uint8_t* p, uint32_t v)
{
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
static void put_u16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static uint32_t get_u32(const uint8_t* p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
static uint32_t get_u16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }

/* Length of the run of equal bytes starting at b[i]. */
static size_t run_length(const uint8_t* b, size_t n, size_t i)
{
    size_t j = i;
    while (j < n && b[j] == b[i]) ++j;
    return j - i;
}

/* Run-length code one byte stream.  Runs of three or more equal bytes become
 * repeat tokens (control 128 + len - 1, then the byte; at most 128 per token,
 * full tokens first); all other bytes are gathered into maximal literal spans
 * (control len - 1, then the bytes; at most 128 per token, full tokens first).
 * Returns the number of bytes written. */
static size_t encode_stream(const uint8_t* b, size_t n, uint8_t* out)
{
    size_t o = 0, i = 0;
    while (i < n) {
        size_t L = run_length(b, n, i);
        if (L >= 3) {
            size_t left = L;
            while (left > 0) {
                size_t piece = left >= 128 ? 128 : left;
                out[o++] = (uint8_t)(128 + piece - 1);
                out[o++] = b[i];
                left -= piece;
            }
            i += L;
        } else {
            size_t start = i;
            while (i < n) {
                size_t r = run_length(b, n, i);
                if (r >= 3) break;
                i += r;
            }
            size_t m = i - start, done = 0;
            while (done < m) {
                size_t piece = (m - done) >= 128 ? 128 : (m - done);
                out[o++] = (uint8_t)(piece - 1);
                memcpy(out + o, b + start + done, piece);
                o += piece;
                done += piece;
            }
        }
    }
    return o;
}

/* Thesis 5.5.1, basic RLE ("mode 0"): 64-bit tokens that compare two RGBA8
 * pixels at once.  A chunk's elements are taken in pairs (element 2k in the
 * low four bytes of unit k, 2k+1 in the high four); runs of two or more equal
 * units become repeat tokens (control 128 + len - 1, then the unit's 8 bytes;
 * at most 128 units per token, full tokens first); the other units form
 * maximal literal spans (control len - 1, then len units of 8 bytes; at most
 * 128 per token, full tokens first).  A chunk of odd length ends with its last
 * element's 4 bytes after the tokens.  Returns the bytes written. */
static size_t encode_units(const uint32_t* e, size_t len, uint8_t* out)
{
    size_t nu = len / 2, o = 0, i = 0;
    while (i < nu) {
        size_t L = 1;
        while (i + L < nu && e[2 * (i + L)] == e[2 * i] && e[2 * (i + L) + 1] == e[2 * i + 1]) ++L;
        if (L >= 2) {
            size_t left = L;
            while (left > 0) {
                size_t piece = left >= 128 ? 128 : left;
                out[o++] = (uint8_t)(128 + piece - 1);
                put_u32(out + o, e[2 * i]);
                put_u32(out + o + 4, e[2 * i + 1]);
                o += 8;
                left -= piece;
            }
            i += L;
        } else {
            size_t start = i;
            /* a unit is literal when it equals neither neighbour */
            while (i < nu && !(i + 1 < nu && e[2 * (i + 1)] == e[2 * i] && e[2 * (i + 1) + 1] == e[2 * i + 1]))
                ++i;
            size_t m = i - start, done = 0;
            while (done < m) {
                size_t piece = (m - done) >= 128 ? 128 : (m - done);
                out[o++] = (uint8_t)(piece - 1);
                for (size_t k = 0; k < piece; ++k) {
                    put_u32(out + o, e[2 * (start + done + k)]);
                    put_u32(out + o + 4, e[2 * (start + done + k) + 1]);
                    o += 8;
                }
                done += piece;
            }
        }
    }
    if (len & 1) {
        put_u32(out + o, e[len - 1]);
        o += 4;
    }
    return o;
}

int64_t orc_rle_compress(const uint32_t* src, int32_t w, int32_t h, int32_t pitch,
                         uint32_t mode, uint8_t* dst, size_t capacity)
{
    if (w < 0 || h < 0 || pitch < w || mode > 2) return -ORC_EINVAL;
    uint64_t n = (uint64_t)w * (uint64_t)h;
    if (n > ORC_MAX_ELEMS) return -ORC_EINVAL;
    if (capacity < orc_rle_max_size(w, h)) return -ORC_ECAP;
    uint64_t nc = n_chunks_of(n);

    put_u32(dst + 0, ORC_MAGIC);
    put_u16(dst + 4, ORC_VERSION);
    put_u16(dst + 6, mode);
    put_u32(dst + 8, (uint32_t)w);
    put_u32(dst + 12, (uint32_t)h);
    put_u32(dst + 16, 4u);
    put_u32(dst + 20, ORC_CHUNK);
    put_u32(dst + 24, (uint32_t)nc);
    put_u32(dst + 28, mode == 0 ? 1u : 4u);

    if (mode == 0) {                    /* one stream per chunk */
        uint8_t* table = dst + ORC_HEADER;
        uint8_t* payload = table + 4u * nc;
        uint32_t e[ORC_CHUNK];
        size_t off = 0;
        for (uint64_t c = 0; c < nc; ++c) {
            uint64_t q0 = c * ORC_CHUNK;
            uint64_t len = (q0 + ORC_CHUNK <= n) ? ORC_CHUNK : n - q0;
            for (uint64_t t = 0; t < len; ++t) {
                uint64_t q = q0 + t;
                e[t] = src[(q / (uint64_t)w) * (uint64_t)pitch + q % (uint64_t)w];
            }
            off += encode_units(e, (size_t)len, payload + off);
            put_u32(table + 4u * c, (uint32_t)off);
        }
        return (int64_t)(ORC_HEADER + 4u * nc + off);
    }

    uint8_t* table = dst + ORC_HEADER;
    uint8_t* payload = table + 16u * nc;
    uint8_t plane[ORC_CHUNK];
    size_t off = 0;
    for (uint64_t c = 0; c < nc; ++c) {
        uint64_t q0 = c * ORC_CHUNK;
        uint64_t len = (q0 + ORC_CHUNK <= n) ? ORC_CHUNK : n - q0;
        for (uint32_t p = 0; p < 4; ++p) {
            for (uint64_t t = 0; t < len; ++t) {
                uint64_t q = q0 + t;
                uint64_t y = q / (uint64_t)w, x = q % (uint64_t)w;
                uint32_t v = src[y * (uint64_t)pitch + x];
                if (mode == 2) v = orc_swizzle(v);
                plane[t] = (uint8_t)(v >> (8 * p));
            }
            off += encode_stream(plane, (size_t)len, payload + off);
            put_u32(table + 4u * (4u * c + p), (uint32_t)off);
        }
    }
    return (int64_t)(ORC_HEADER + 16u * nc + off);
}

int orc_rle_decompress(const uint8_t* src, size_t size, uint32_t* dst,
                       int32_t w, int32_t h, int32_t pitch)
{
    if (w < 0 || h < 0 || pitch < w) return ORC_EINVAL;
    if (!src || size < ORC_HEADER) return ORC_ECORRUPT;
    if (get_u32(src) != ORC_MAGIC || get_u16(src + 4) != ORC_VERSION) return ORC_ECORRUPT;
    uint32_t mode = get_u16(src + 6);
    if (mode > 2) return ORC_ECORRUPT;
    if (get_u32(src + 8) != (uint32_t)w || get_u32(src + 12) != (uint32_t)h) return ORC_ECORRUPT;
    if (get_u32(src + 16) != 4u || get_u32(src + 20) != ORC_CHUNK || get_u32(src + 28) != (mode == 0 ? 1u : 4u))
        return ORC_ECORRUPT;
    uint64_t n = (uint64_t)w * (uint64_t)h;
    uint64_t nc = n_chunks_of(n);
    if (get_u32(src + 24) != nc) return ORC_ECORRUPT;
    if (mode == 0) {
        if (size < ORC_HEADER + 4u * nc) return ORC_ECORRUPT;
        const uint8_t* table = src + ORC_HEADER;
        const uint8_t* payload = table + 4u * nc;
        size_t payload_size = size - (ORC_HEADER + 4u * nc);
        size_t begin = 0;
        for (uint64_t c = 0; c < nc; ++c) {
            uint64_t q0 = c * ORC_CHUNK;
            size_t len = (size_t)((q0 + ORC_CHUNK <= n) ? ORC_CHUNK : n - q0), nu = len / 2;
            size_t end = get_u32(table + 4u * c);
            if (end < begin || end > payload_size) return ORC_ECORRUPT;
            /* no valid stream is longer than the all-literal coding of its chunk */
            if (end - begin > 8 * nu + (nu + 127) / 128 + 4 * (len & 1)) return ORC_ECORRUPT;
            uint32_t e[ORC_CHUNK];
            size_t i = begin, o = 0;     /* o counts units */
            while (o < nu) {
                if (i >= end) return ORC_ECORRUPT;
                uint32_t ctl = payload[i++];
                size_t m = ctl < 128 ? ctl + 1 : ctl - 127;
                if (o + m > nu) return ORC_ECORRUPT;
                if (ctl < 128) {
                    if (i + 8 * m > end) return ORC_ECORRUPT;
                    for (size_t k = 0; k < m; ++k) {
                        e[2 * (o + k)] = get_u32(payload + i + 8 * k);
                        e[2 * (o + k) + 1] = get_u32(payload + i + 8 * k + 4);
                    }
                    i += 8 * m;
                } else {
                    if (i + 8 > end) return ORC_ECORRUPT;
                    for (size_t k = 0; k < m; ++k) {
                        e[2 * (o + k)] = get_u32(payload + i);
                        e[2 * (o + k) + 1] = get_u32(payload + i + 4);
                    }
                    i += 8;
                }
                o += m;
            }
            if (len & 1) {
                if (i + 4 > end) return ORC_ECORRUPT;
                e[len - 1] = get_u32(payload + i);
                i += 4;
            }
            if (i != end) return ORC_ECORRUPT;
            for (size_t t = 0; t < len; ++t) {
                uint64_t q = q0 + t;
                dst[(q / (uint64_t)w) * (uint64_t)pitch + q % (uint64_t)w] = e[t];
            }
            begin = end;
        }
        return ORC_OK;
    }
    if (size < ORC_HEADER + 16u * nc) return ORC_ECORRUPT;
    const uint8_t* table = src + ORC_HEADER;
    const uint8_t* payload = table + 16u * nc;
    size_t payload_size = size - (ORC_HEADER + 16u * nc);

    uint8_t planes[4][ORC_CHUNK];
    size_t begin = 0;
    for (uint64_t c = 0; c < nc; ++c) {
        uint64_t q0 = c * ORC_CHUNK;
        size_t len = (size_t)((q0 + ORC_CHUNK <= n) ? ORC_CHUNK : n - q0);
        for (uint32_t p = 0; p < 4; ++p) {
            size_t end = get_u32(table + 4u * (4u * c + p));
            if (end < begin || end > payload_size) return ORC_ECORRUPT;
            /* no valid stream is longer than the all-literal coding of its chunk */
            if (end - begin > len + (len + 127) / 128) return ORC_ECORRUPT;
            /* decode: control < 128 copies control+1 bytes, otherwise the next
             * byte repeats control-127 times */
            size_t i = begin, o = 0;
            while (i < end) {
                uint32_t ctl = payload[i++];
                if (ctl < 128) {
                    size_t m = ctl + 1;
                    if (i + m > end || o + m > len) return ORC_ECORRUPT;
                    memcpy(planes[p] + o, payload + i, m);
                    i += m;
                    o += m;
                } else {
                    size_t m = ctl - 127;
                    if (i + 1 > end || o + m > len) return ORC_ECORRUPT;
                    memset(planes[p] + o, payload[i], m);
                    i += 1;
                    o += m;
                }
            }
            if (o != len) return ORC_ECORRUPT;
            begin = end;
        }
        for (size_t t = 0; t < len; ++t) {
            uint32_t v = (uint32_t)planes[0][t] | ((uint32_t)planes[1][t] << 8) |
                         ((uint32_t)planes[2][t] << 16) | ((uint32_t)planes[3][t] << 24);
            if (mode == 2) v = orc_unswizzle(v);
            uint64_t q = q0 + t;
            uint64_t y = q / (uint64_t)w, x = q % (uint64_t)w;
            dst[y * (uint64_t)pitch + x] = v;
        }
    }
    return ORC_OK;
}

/* ---- lossy YUV compressor (thesis 5.5.3) ------------------------------- */

/* Colour-space conversion and chroma subsampling before run-length coding.
 * The thesis names the steps but prints no formulas; this is the full-range
 * BT.601 (JFIF) transform in 8-bit fixed point (coefficients x 256):
 *   Y = (77 R + 150 G + 29 B + 128) / 256
 *   U = 128 + (-43 R - 85 G + 128 B + 128) / 256      (clamped to 255)
 *   V = 128 + (128 R - 107 G - 21 B + 128) / 256      (clamped to 255)
 * with divisions rounding down.  Every 2x2 block keeps its four Y values and
 * the rounded means of its pixels' U, V and alpha (over the pixels the image
 * has).  Packed image: ceil(w/2) x 2 ceil(h/2) words; row by of the top half
 * holds the blocks' luma words (byte k = Y of pixel (2bx + (k & 1),
 * 2by + (k >> 1)), 0 where the image has no pixel), row ceil(h/2) + by the
 * chroma words (bytes U, V, A, 0).  Decoding gives every pixel its block's
 * U, V and alpha:
 *   R = Y + (359 (V-128) + 128) / 256,  G = Y - (88 (U-128) + 183 (V-128) + 128) / 256,
 *   B = Y + (454 (U-128) + 128) / 256,  each clamped to [0, 255]. */
static int32_t floor_div256(int32_t x) { return x >= 0 ? x / 256 : -((-x + 255) / 256); }
static int32_t clamp255(int32_t v) { return v < 0 ? 0 : (v > 255 ? 255 : v); }

int orc_yuv_encode(const uint32_t* src, int32_t w, int32_t h, int32_t pitch, uint32_t* dst)
{
    if (w < 0 || h < 0 || pitch < w) return ORC_EINVAL;
    int32_t bw = (w + 1) / 2, bh = (h + 1) / 2;
    for (int32_t by = 0; by < bh; ++by) {
        for (int32_t bx = 0; bx < bw; ++bx) {
            uint32_t luma = 0;
            int32_t su = 0, sv = 0, sa = 0, cnt = 0;
            for (int k = 0; k < 4; ++k) {
                int32_t x = 2 * bx + (k & 1), y = 2 * by + (k >> 1);
                if (x >= w || y >= h) continue;
                uint32_t v = src[(size_t)y * pitch + x];
                int32_t R = v & 0xFF, G = (v >> 8) & 0xFF, B = (v >> 16) & 0xFF, A = (int32_t)(v >> 24);
                int32_t Y = floor_div256(77 * R + 150 * G + 29 * B + 128);
                int32_t U = clamp255(128 + floor_div256(-43 * R - 85 * G + 128 * B + 128));
                int32_t V = clamp255(128 + floor_div256(128 * R - 107 * G - 21 * B + 128));
                luma |= (uint32_t)Y << (8 * k);
                su += U;
                sv += V;
                sa += A;
                ++cnt;
            }
            dst[(size_t)by * bw + bx] = luma;
            dst[(size_t)(bh + by) * bw + bx] = (uint32_t)((su + cnt / 2) / cnt) |
                                               ((uint32_t)((sv + cnt / 2) / cnt) << 8) |
                                               ((uint32_t)((sa + cnt / 2) / cnt) << 16);
        }
    }
    return ORC_OK;
}

int orc_yuv_decode(const uint32_t* src, int32_t w, int32_t h, uint32_t* dst, int32_t pitch)
{
    if (w < 0 || h < 0 || pitch < w) return ORC_EINVAL;
    int32_t bw = (w + 1) / 2, bh = (h + 1) / 2;
    for (int32_t y = 0; y < h; ++y) {
        for (int32_t x = 0; x < w; ++x) {
            int32_t bx = x / 2, by = y / 2, k = (x & 1) + 2 * (y & 1);
            uint32_t luma = src[(size_t)by * bw + bx], ch = src[(size_t)(bh + by) * bw + bx];
            int32_t Y = (luma >> (8 * k)) & 0xFF;
            int32_t U = (int32_t)(ch & 0xFF) - 128, V = (int32_t)((ch >> 8) & 0xFF) - 128;
            int32_t A = (ch >> 16) & 0xFF;
            int32_t R = clamp255(Y + floor_div256(359 * V + 128));
            int32_t G = clamp255(Y - floor_div256(88 * U + 183 * V + 128));
            int32_t B = clamp255(Y + floor_div256(454 * U + 128));
            dst[(size_t)y * pitch + x] = (uint32_t)R | ((uint32_t)G << 8) | ((uint32_t)B << 16) | ((uint32_t)A << 24);
        }
    }
    return ORC_OK;
}

/* ---- automatic region of interest (thesis 5.3) ------------------------- */

static int holds_data(int32_t format, const void* color, const float* depth, size_t e)
{
    if (depth) return depth[e] < 1.0f;
    if (format == 0) return ((const uint32_t*)color)[e] != 0u;
    if (format == 1) {
        const float* f = (const float*)color + 4 * e;
        return f[0] != 0.0f || f[1] != 0.0f || f[2] != 0.0f || f[3] != 0.0f;
    }
    const uint16_t* h = (const uint16_t*)color + 4 * e;
    return (h[0] & 0x7FFFu) || (h[1] & 0x7FFFu) || (h[2] & 0x7FFFu) || (h[3] & 0x7FFFu);
}

int orc_detect_roi(orc_rect pvp, orc_rect search, int32_t pitch, int32_t format,
                   const void* color, const float* depth, int32_t tile, uint8_t* occ,
                   orc_rect* roi)
{
    if (pvp.w < 0 || pvp.h < 0 || pitch < pvp.w || tile < 1 || !roi) return ORC_EINVAL;
    if (!depth && (format < 0 || format > 2)) return ORC_EINVAL;
    int64_t gw = (pvp.w + tile - 1) / tile, gh = (pvp.h + tile - 1) / tile;
    if (occ) memset(occ, 0, (size_t)(gw * gh));
    /* the examined pixels: search clipped to pvp, relative to the pvp origin */
    int64_t x0 = (int64_t)search.x - pvp.x, y0 = (int64_t)search.y - pvp.y;
    int64_t x1 = x0 + search.w, y1 = y0 + search.h;
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > pvp.w) x1 = pvp.w;
    if (y1 > pvp.h) y1 = pvp.h;
    int have = 0;
    int64_t bx0 = 0, by0 = 0, bx1 = 0, by1 = 0;
    for (int64_t y = y0; y < y1; ++y) {
        for (int64_t x = x0; x < x1; ++x) {
            if (!holds_data(format, color, depth, (size_t)(y * pitch + x))) continue;
            if (!have) { bx0 = bx1 = x; by0 = by1 = y; have = 1; }
            if (x < bx0) bx0 = x;
            if (x > bx1) bx1 = x;
            if (y < by0) by0 = y;
            if (y > by1) by1 = y;
            if (occ) occ[(y / tile) * gw + x / tile] = 1;
        }
    }
    if (!have) {
        roi->x = roi->y = roi->w = roi->h = 0;
        return ORC_OK;
    }
    roi->x = (int32_t)(pvp.x + bx0);
    roi->y = (int32_t)(pvp.y + by0);
    roi->w = (int32_t)(bx1 - bx0 + 1);
    roi->h = (int32_t)(by1 - by0 + 1);
    return ORC_OK;
}

/* ---- assembly of the other compound modes (thesis 4.2) ----------------- */

static int in_rect(orc_rect r, int64_t x, int64_t y)
{
    return x >= r.x && x < (int64_t)r.x + r.w && y >= r.y && y < (int64_t)r.y + r.h;
}

int orc_assemble_tiles(const orc_layer* src, int32_t n, int32_t bpp, orc_rect out_pvp,
                       int32_t out_pitch, void* out)
{
    if (n < 0 || (bpp != 4 && bpp != 8 && bpp != 16) || out_pitch < out_pvp.w) return ORC_EINVAL;
    uint8_t* o = (uint8_t*)out;
    for (int32_t i = 0; i < n; ++i) {
        const orc_layer* s = &src[i];
        for (int64_t py = out_pvp.y; py < (int64_t)out_pvp.y + out_pvp.h; ++py) {
            for (int64_t px = out_pvp.x; px < (int64_t)out_pvp.x + out_pvp.w; ++px) {
                if (!in_rect(s->roi, px, py) || !in_rect(s->pvp, px, py)) continue;
                const size_t e = (size_t)((py - s->pvp.y) * s->pitch + (px - s->pvp.x));
                const size_t d = (size_t)((py - out_pvp.y) * out_pitch + (px - out_pvp.x));
                memcpy(o + d * bpp, (const uint8_t*)s->color + e * bpp, (size_t)bpp);
            }
        }
    }
    return ORC_OK;
}

int orc_assemble_pixels(const void* const* src, const int32_t* pitch, const int32_t* kx,
                        const int32_t* ky, int32_t n, int32_t nx, int32_t ny, int32_t bpp,
                        orc_rect out_pvp, int32_t out_pitch, void* out)
{
    if (n < 0 || nx < 1 || ny < 1 || (bpp != 4 && bpp != 8 && bpp != 16) || out_pitch < out_pvp.w)
        return ORC_EINVAL;
    uint8_t* o = (uint8_t*)out;
    for (int32_t k = 0; k < n; ++k) {
        if (kx[k] < 0 || kx[k] >= nx || ky[k] < 0 || ky[k] >= ny) return ORC_EINVAL;
        const int64_t w = out_pvp.w > kx[k] ? (out_pvp.w - kx[k] + nx - 1) / nx : 0;
        const int64_t h = out_pvp.h > ky[k] ? (out_pvp.h - ky[k] + ny - 1) / ny : 0;
        if (pitch[k] < w) return ORC_EINVAL;
        for (int64_t j = 0; j < h; ++j) {
            for (int64_t i = 0; i < w; ++i) {
                const int64_t dx = kx[k] + i * nx, dy = ky[k] + j * ny;
                memcpy(o + (size_t)(dy * out_pitch + dx) * bpp,
                       (const uint8_t*)src[k] + (size_t)(j * pitch[k] + i) * bpp, (size_t)bpp);
            }
        }
    }
    return ORC_OK;
}

int orc_average(const orc_layer* src, int32_t n, int32_t format, orc_rect out_pvp,
                int32_t out_pitch, void* out)
{
    if (n < 0 || (format != 0 && format != ORC_F32 && format != ORC_F16) || out_pitch < out_pvp.w)
        return ORC_EINVAL;
    for (int64_t py = out_pvp.y; py < (int64_t)out_pvp.y + out_pvp.h; ++py) {
        for (int64_t px = out_pvp.x; px < (int64_t)out_pvp.x + out_pvp.w; ++px) {
            const size_t d = (size_t)((py - out_pvp.y) * out_pitch + (px - out_pvp.x));
            uint64_t isum[4] = {0, 0, 0, 0};
            double fsum[4] = {0.0, 0.0, 0.0, 0.0};
            int64_t count = 0;
            for (int32_t i = 0; i < n; ++i) {
                const orc_layer* s = &src[i];
                if (!in_rect(s->roi, px, py) || !in_rect(s->pvp, px, py)) continue;
                const size_t e = (size_t)((py - s->pvp.y) * s->pitch + (px - s->pvp.x));
                ++count;
                for (int ch = 0; ch < 4; ++ch) {
                    if (format == 0) isum[ch] += (((const uint32_t*)s->color)[e] >> (8 * ch)) & 0xFFu;
                    else if (format == ORC_F32) fsum[ch] += ((const float*)s->color)[4 * e + ch];
                    else fsum[ch] += half_to_double(((const uint16_t*)s->color)[4 * e + ch]);
                }
            }
            if (format == 0) {
                uint32_t v = 0;
                for (int ch = 0; ch < 4; ++ch)
                    if (count) v |= (uint32_t)((isum[ch] + (uint64_t)count / 2) / (uint64_t)count) << (8 * ch);
                ((uint32_t*)out)[d] = v;
            } else {
                for (int ch = 0; ch < 4; ++ch) ((double*)out)[4 * d + ch] = count ? fsum[ch] / (double)count : 0.0;
            }
        }
    }
    return ORC_OK;
}
