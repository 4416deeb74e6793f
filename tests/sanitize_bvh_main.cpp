// Host BVH build and host walk under AddressSanitizer / UndefinedBehaviorSanitizer, and under
// ThreadSanitizer for the build's worker threads (tests/test_sanitizers.py compiles this with the
// library's host build source).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
#include <vector>

#include "gsp_internal.h"

static int check(const char* what, bool ok) {
    if (!ok) std::fprintf(stderr, "FAILED: %s\n", what);
    return ok ? 0 : 1;
}

int main() {
    int bad = 0;
    std::mt19937 rng(7);
    std::uniform_real_distribution<float> u(-1.0f, 1.0f);
    // 70,001 triangles take the multi-threaded build (worker threads over subtrees and link sets)
    for (int nt : {1, 2, 3, 17, 500, 4099, 70001}) {
        std::vector<float> v(9 * (size_t)nt);
        std::vector<int32_t> t(3 * (size_t)nt);
        for (int i = 0; i < nt; ++i) {
            const float cx = u(rng), cy = u(rng), cz = u(rng);
            for (int k = 0; k < 3; ++k) {
                v[9 * i + 3 * k] = cx + 0.05f * u(rng);
                v[9 * i + 3 * k + 1] = cy + 0.05f * u(rng);
                v[9 * i + 3 * k + 2] = nt == 17 ? 0.5f : cz + 0.05f * u(rng);  // one planar case
                t[3 * i + k] = 3 * i + k;
            }
        }
        for (int sets : {1, 6}) {
            gsp_bvh_params p{16, 4, 7, sets};
            HostBVH b;
            const std::string err = bvh_build_host(v.data(), 3 * (int64_t)nt, t.data(), nt, p, b);
            bad += check("build", err.empty());
            bad += check("node count", b.nnodes >= 1 && (int64_t)b.nodes.size() == sets * b.stride * 2);
            const int n = 257;
            std::vector<float> rays(8 * n);
            for (int i = 0; i < n; ++i) {
                float d[3] = {u(rng), u(rng), u(rng)};
                const float l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) + 1e-6f;
                const float r[8] = {2 * u(rng), 2 * u(rng), 2 * u(rng), 0.0f, d[0] / l, d[1] / l, d[2] / l, INFINITY};
                std::memcpy(&rays[8 * i], r, sizeof r);
            }
            std::vector<int32_t> tri(n), vis(n), tests(n);
            std::vector<float> tt(n);
            bvh_host_walk(b, rays.data(), n, tri.data(), tt.data(), vis.data(), tests.data());
            for (int i = 0; i < n; ++i) bad += check("hit index", tri[i] >= -1 && tri[i] < nt);
        }
    }
    // degenerate: every triangle at the same centroid, and a zero-area triangle
    std::vector<float> v(9 * 64, 0.25f);
    std::vector<int32_t> t(3 * 64);
    for (int i = 0; i < 3 * 64; ++i) t[i] = i;
    gsp_bvh_params p{16, 4, 7, 6};
    HostBVH b;
    bad += check("degenerate build", bvh_build_host(v.data(), 3 * 64, t.data(), 64, p, b).empty());
    std::printf(bad ? "sanitized host build: %d failures\n" : "sanitized host build: ok\n", bad);
    return bad ? 1 : 0;
}
