/* Drives the FP64 oracle through its frame-level entry points on small synthetic inputs, for a
 * build with AddressSanitizer and UndefinedBehaviorSanitizer (tests/test_oracle_sanitized.py):
 * every buffer access, allocation and free of the row-window, model-order, 2-D band, square-block
 * and unwrapping paths runs once under the sanitizers. Exits 0 and prints "ok" when every call
 * returns its documented success value; a sanitizer report aborts with a non-zero status. */
#include "../oracle/rmusic_oracle.c"

#include <stdio.h>

static uint32_t lcg_state = 12345u;
static double noise(void) { /* uniform in [-0.5, 0.5) */
    lcg_state = lcg_state * 1664525u + 1013904223u;
    return (double)(lcg_state >> 8) / 16777216.0 - 0.5;
}

static int check(const char* what, int rc) {
    if (rc < 0) {
        printf("%s returned %d\n", what, rc);
        return 1;
    }
    return 0;
}

int main(void) {
    enum { H = 40, W = 160 };
    static float img[H * W];
    static uint16_t img16[H * W];
    static double cimg[2 * H * W];
    static double out[H * W], dx[H * W], dy[H * W], al[H * W], unw[H * W];
    static uint8_t st[H * W];
    static float wrapped[H * W];
    static int32_t kk[H * W];
    int bad = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const double r2 = (x - 80.0) * (x - 80.0) + (y - 20.0) * (y - 20.0);
            const double phi = 2.5 * exp(-r2 / 300.0);
            const double v = 0.5 + 0.4 * cos(2.0 * ORC_PI * 0.1 * x + phi) + 0.01 * noise();
            img[y * W + x] = (float)v;
            img16[y * W + x] = (uint16_t)lround(4095.0 * (v < 0 ? 0 : v > 1 ? 1 : v));
            cimg[2 * (y * W + x)] = cos(phi + 0.3 * x) + 0.05 * noise();
            cimg[2 * (y * W + x) + 1] = sin(phi + 0.3 * x) + 0.05 * noise();
            const double w = fmod(phi * 3.0 + 0.05 * x + ORC_PI, 2.0 * ORC_PI) - ORC_PI;
            wrapped[y * W + x] = (float)w;
        }
    orc_params p = {32, 8, 1, 1, 0, 0, 0.1, 0.0, 0.0, 0};
    bad |= check("rows fb", orc_demodulate(img, ORC_F32, H, W, &p, out, st, 1));
    p.deriv_axis = 1;
    bad |= check("columns uint16", orc_demodulate(img16, ORC_U16, H, W, &p, out, st, 1));
    p.deriv_axis = 0;
    p.forward_backward = 0;
    p.window_len = 12;
    p.cov_order = 3;
    bad |= check("forward only L=3", orc_demodulate(img, ORC_F32, H, W, &p, out, st, 1));
    p.forward_backward = 1;
    p.window_len = 32;
    p.cov_order = 8;
    p.band_cross = 0.1;
    bad |= check("2-D band", orc_demodulate(img, ORC_F32, H, W, &p, out, st, 1));
    p.band_cross = 0.0;
    p.raw_input = 1;
    p.model_order = 2;
    bad |= check("model order 2, raw", orc_demodulate(img, ORC_F32, H, W, &p, out, st, 1));
    p.raw_input = 0;
    p.model_order = 1;
    p.carrier_freq = 0.0;
    bad |= check("square block", orc_square_demodulate(cimg, ORC_C128, H, W, &p, 3, dx, dy, al, st, 1));
    bad |= check("unwrap", orc_unwrap(wrapped, H, W, unw, kk));
    if (bad) return 1;
    printf("ok\n");
    return 0;
}
