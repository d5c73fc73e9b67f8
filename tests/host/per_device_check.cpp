// Host-side checks of the engine's internal helpers (no GPU): the per-device
// set-up record keeps each device's state apart, and the triangular tile
// numbering inverts exactly.  Prints "ok" and exits 0 on success.
#include <cstdio>

#include "krr_internal.h"

static krr::PerDevice g_rec;  // static storage: zero-initialised, as in the library

int main() {
    using krr::PerDevice;
    // a set-up done on device 0 must not count for device 1, and the values
    // (cluster counts) stay per device
    if (g_rec.has(0) || g_rec.has(1)) return 1;
    g_rec.put(0, 36);
    if (!g_rec.has(0) || g_rec.has(1) || g_rec.get(0) != 36) return 2;
    g_rec.put(1, 38);
    if (!g_rec.has(1) || g_rec.get(1) != 38 || g_rec.get(0) != 36) return 3;
    // out-of-range devices are never recorded (set up on every call)
    g_rec.put(krr::MAX_DEVICES, 5);
    g_rec.put(-1, 5);
    if (g_rec.has(krr::MAX_DEVICES) || g_rec.has(-1)) return 4;
    // tri_decode inverts tri_index, including indices past 2^24 where the
    // single-precision estimate is off
    const int64_t rows[] = {0, 1, 2, 7, 127, 4095, 8191, 65535, 131071};
    for (int64_t i : rows)
        for (int64_t j : {int64_t(0), i / 2, i}) {
            int64_t a = -1, b = -1;
            krr::tri_decode(krr::tri_index(i, j), &a, &b);
            if (a != i || b != j) {
                std::printf("tri_decode(%lld, %lld) -> (%lld, %lld)\n", (long long)i, (long long)j, (long long)a,
                            (long long)b);
                return 5;
            }
        }
    std::printf("ok\n");
    return 0;
}
