// Host-only probe of the single-launch attempt planner (attempt_small.h): for
// meshes "nx ny" read from stdin (one plane), prints one JSON object with the
// eligibility and, per cluster size, the rows and column units of every CTA and
// the shared-memory layout in both precisions.  Launches nothing and makes no
// CUDA call.
#include <cstdio>
#include <cstring>

#include "attempt_small.h"
#include "plan.h"

using namespace mm;

int main() {
    int nx, ny;
    while (scanf("%d %d", &nx, &ny) == 2) {
        SimDesc d;
        memset(&d, 0, sizeof(d));
        d.nx = nx; d.ny = ny; d.nz = 1;
        d.ncells = nx * ny;
        d.flags = F_DEMAG;
        d.group_begin = -1;
        plan_geometry(d, true);
        printf("{\"mesh\": [%d,%d], \"Px\": %d, \"Py\": %d, \"Kx\": %d, \"eligible\": %d, \"halves\": %d, \"nc\": {",
               nx, ny, d.Px, d.Py, d.Kx, small_eligible(d) ? 1 : 0, small_halves(d));
        for (int nc = 1, first = 1; nc <= kSmallMaxCluster; nc <<= 1, first = 0) {
            printf("%s\"%d\": {\"rb\": %d, \"cu\": %d", first ? "" : ", ", nc, small_rows_per_cta(d, nc),
                   small_units_per_cta(d, nc));
            const size_t sz[2][2] = {{4, 4}, {8, 8}};
            const char* nm[2] = {"f32", "f64"};
            for (int k = 0; k < 2; ++k) {
                const SmallLayout L = small_layout(d, nc, sz[k][0], sz[k][1]);
                printf(", \"%s\": [%zu,%zu,%zu,%zu,%zu,%zu,%zu]", nm[k], L.halo, L.colin, L.spec, L.rowin, L.w64,
                       L.tens, L.total);
            }
            printf("}");
        }
        printf("}}\n");
    }
    return 0;
}
