// Test driver for the plan-time entry ordering of the balanced gridding kernel
// (order_warp_entries in the library's plan.cpp), built by test_host_logic.py with
// the host compiler: no GPU and no CUDA runtime calls.
//
// stdin:  number of groups; per group "members nmax" then, per member lane, "n e_0 .. e_{n-1}"
// stdout: per group one line of 32 * nmax "element payload" pairs (entry k of lane l at
//         index 32 k + l); a real entry's payload is 1 + its position in the lane's input list,
//         a padding entry's payload is 0.
#include <cstdio>
#include <vector>

#include "epic_internal.h"

int main()
{
    int ngroups = 0;
    if (std::scanf("%d", &ngroups) != 1) return 1;
    for (int g = 0; g < ngroups; ++g) {
        int members = 0, nmax = 0;
        if (std::scanf("%d %d", &members, &nmax) != 2) return 1;
        std::vector<std::vector<int2>> cells(members);
        for (int l = 0; l < members; ++l) {
            int n = 0;
            if (std::scanf("%d", &n) != 1) return 1;
            for (int i = 0; i < n; ++i) {
                int e = 0;
                if (std::scanf("%d", &e) != 1) return 1;
                cells[l].push_back(make_int2(e, i + 1));
            }
        }
        std::vector<int2> out(32 * (size_t)nmax, make_int2(-1, -1));
        epic::order_warp_entries(cells, nmax, out.data());
        for (const int2& en : out) std::printf("%d %d ", en.x, en.y);
        std::printf("\n");
    }
    return 0;
}
