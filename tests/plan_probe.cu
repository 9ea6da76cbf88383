// Host-only probe of the simulation planner (plan.h): reads meshes
// "nx ny nz f32" from stdin and prints one JSON object per mesh with the padded
// sizes, tile shapes, work lists and shared-memory sizes; then prints the term
// flags plan_coefficients / plan_extended give a set of materials.  Launches
// nothing and makes no CUDA call.
#include <cstdio>
#include <cstring>

#include "plan.h"

using namespace mm;

static void print_items(const char* name, const std::vector<WorkItem>& v) {
    printf("\"%s\": [", name);
    for (size_t i = 0; i < v.size(); ++i) printf("%s[%d,%d,%d,%d]", i ? "," : "", v[i].sim, v[i].a, v[i].b, v[i].c);
    printf("]");
}

int main() {
    int nx, ny, nz, f32;
    while (scanf("%d %d %d %d", &nx, &ny, &nz, &f32) == 4) {
        SimDesc d;
        memset(&d, 0, sizeof(d));
        d.nx = nx; d.ny = ny; d.nz = nz;
        d.ncells = nx * ny * nz;
        d.flags = F_DEMAG;
        plan_geometry(d, f32 != 0);
        PlanItems P;
        const size_t vsz = f32 ? 8 : 16;
        plan_items(d, 0, vsz, P);
        printf("{\"mesh\": [%d,%d,%d], \"f32\": %d, \"Px\": %d, \"Py\": %d, \"Pz\": %d, \"Kx\": %d, \"Rx\": %d, "
               "\"Ty\": %d, \"NBx\": %d, \"ncomp\": %d, \"yzc\": %d, \"yzc_list\": %d, \"tens\": %lld, \"spec\": %lld, ",
               nx, ny, nz, f32, d.Px, d.Py, d.Pz, d.Kx, d.Rx, d.Ty, d.NBx, d.ncomp, plan_uses_yzc(d) ? 1 : 0,
               plan_uses_yzc(d) ? plan_yzc_list(d, f32 != 0) : -1, plan_tens_elems(d), plan_spec_elems(d));
        printf("\"smem\": [%zu,%zu,%zu,%zu,%zu,%zu], ", P.smem_x, P.smem_xi, P.smem_y13, P.smem_z, P.smem_y2,
               P.smem_yzc);
        print_items("x", P.x); printf(", ");
        print_items("y13", P.y13); printf(", ");
        print_items("z", P.z); printf(", ");
        print_items("y2", P.y2); printf(", ");
        std::vector<WorkItem> all;
        for (int li = 0; li < kYzcListCount; ++li) all.insert(all.end(), P.yzc[li].begin(), P.yzc[li].end());
        print_items("yzc_items", all);
        // autotuner candidates of each phase, starting from the rule
        Tuning fixed;
        fixed.Ty = d.Ty;
        fixed.Rx = d.Rx;
        fixed.col_group = (f32 && plan_uses_yzc(d)) ? (plan_yzc_wide(plan_yzc_list(d, true)) ? 2 : 1) : 0;
        printf(", \"cands\": [");
        for (int ph = 0; ph < 3; ++ph) {
            const std::vector<Tuning> c = plan_tuning_candidates(d, f32 != 0, ph, fixed);
            printf("%s[", ph ? "," : "");
            for (size_t i = 0; i < c.size(); ++i) {
                SimDesc e = d;
                plan_geometry(e, f32 != 0, c[i]);
                PlanItems Q;
                plan_items(e, 0, vsz, Q);
                printf("%s{\"Ty\": %d, \"Rx\": %d, \"xt\": %d, \"ct\": %d, \"g\": %d, \"occ\": %d, \"st\": %d, \"pTy\": %d, \"pRx\": %d, "
                       "\"smem\": [%zu,%zu,%zu,%zu,%zu,%zu], \"list\": %d}",
                       i ? "," : "", c[i].Ty, c[i].Rx, c[i].x_threads, c[i].col_threads, c[i].col_group, c[i].col_occ, c[i].x_stage, e.Ty, e.Rx,
                       Q.smem_x, Q.smem_xi, Q.smem_y13, Q.smem_z, Q.smem_y2, Q.smem_yzc,
                       plan_uses_yzc(e) ? plan_yzc_list(e, f32 != 0) : -1);
            }
            printf("]");
        }
        printf("]}\n");
    }
    // term flags: (dmi kind, D, A, cells, A cells any, D cells any, u_x, aJ)
    const double cases[][8] = {
        {1, 3e-3, 1e-11, 0, 0, 0, 0, 0}, {1, 0, 1e-11, 0, 0, 0, 0, 0}, {2, 3e-3, 1e-11, 0, 0, 0, 0, 0},
        {3, 3e-3, 0, 0, 0, 0, 0, 0},     {1, 0, 0, 1, 1, 1, 0, 0},     {0, 3e-3, 1e-11, 0, 0, 0, 0, 0},
        {1, 0, 0, 1, 0, 0, 0, 0},        {0, 0, 1e-11, 0, 0, 0, 50, 0}, {0, 0, 1e-11, 0, 0, 0, 0, 1e9},
        {2, 0, 0, 1, 0, 1, 0, 0},
    };
    for (const auto& c : cases) {
        SimDesc d;
        memset(&d, 0, sizeof(d));
        d.nx = d.ny = d.nz = 2;
        d.dx = d.dy = d.dz = 1e-9;
        d.gamma = 2.2e5;
        d.alpha = 0.1;
        d.dmi_kind = (int)c[0];
        d.D = c[1];
        d.A = c[2];
        d.u_stt[0] = c[6];
        d.aJ = c[7];
        d.p[2] = 1.0;
        plan_coefficients(d, d.dmi_kind == 1);
        plan_extended(d, c[3] != 0, c[4] != 0, c[5] != 0);
        printf("{\"flags_case\": [%g,%g,%g,%g,%g,%g,%g,%g], \"flags\": %d, \"eflags\": %d}\n", c[0], c[1], c[2],
               c[3], c[4], c[5], c[6], c[7], d.flags, d.eflags);
    }
    return 0;
}
