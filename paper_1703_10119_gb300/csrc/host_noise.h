// Host side of the noise-table upload: gathering one face's per-wall tables into a contiguous chunk while
// checking every value. Plain C++ without CUDA: the library (hygro_api.cu) includes it, and the CPU tests
// compile it on their own.
#pragma once

#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

namespace hygro {

// Copies pairs [p0, p1) of a face's concatenated tables into dst: the k-th table starts at pair start[k]
// (ascending, start[0] = 0), has len[k] > 0 pairs of floats (T, Pv) and is read from src[k]. Splits the
// range over up to `threads` host threads, no thread taking fewer than min_pairs pairs, each checking the
// values it copies. Returns the index of the first pair holding a non-finite value, or -1.
inline int64_t gather_tables(const std::vector<const float *> &src, const std::vector<int64_t> &start,
                             const std::vector<int64_t> &len, int64_t p0, int64_t p1, float *dst, int threads,
                             int64_t min_pairs = int64_t(1) << 18)
{
    auto part = [&](int64_t a, int64_t b) -> int64_t {
        if (a >= b) return -1;
        size_t k = (size_t)(std::upper_bound(start.begin(), start.end(), a) - start.begin()) - 1;
        int64_t x = a;
        while (x < b) {
            const int64_t s = start[k], e = std::min(b, s + len[k]);
            const float *in = src[k] + 2 * (x - s);
            float *out = dst + 2 * (x - p0);
            const int64_t n = 2 * (e - x);
            uint32_t bad = 0;
            for (int64_t i = 0; i < n; ++i) {   // branch-free copy and check (vectorises)
                uint32_t u;
                memcpy(&u, in + i, sizeof u);
                memcpy(out + i, &u, sizeof u);
                bad |= (uint32_t)((u & 0x7f800000u) == 0x7f800000u);   // exponent all ones: inf or nan
            }
            if (bad)
                for (int64_t i = 0; i < n; ++i)
                    if (!std::isfinite(in[i])) return x + i / 2;
            x = e;
            ++k;
        }
        return -1;
    };
    const int64_t n = p1 - p0;
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(threads, n / std::max<int64_t>(1, min_pairs)));
    std::vector<int64_t> first_bad(T, -1);
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) {
        try {
            pool.emplace_back([&, t] { first_bad[t] = part(p0 + n * t / T, p0 + n * (t + 1) / T); });
        } catch (...) {   // no thread: this part on the calling thread
            first_bad[t] = part(p0 + n * t / T, p0 + n * (t + 1) / T);
        }
    }
    first_bad[0] = part(p0, p0 + n / T);
    for (auto &th : pool) th.join();
    for (int t = 0; t < T; ++t)
        if (first_bad[t] >= 0) return first_bad[t];
    return -1;
}

}  // namespace hygro
