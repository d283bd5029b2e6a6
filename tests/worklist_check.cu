// Host-only harness of the persistent kernel's column work list (worklist.h),
// run by tests/test_worklist.py on the CPU (no CUDA call is made).
// Arguments: G, then one "slot nbx nby nbz bsx bsy bsz ntile" group per mesh.
// Output: one line "slot blk tile z0 z1" per queued item, in queue order.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "worklist.h"

int main(int argc, char** argv) {
    if (argc < 10 || (argc - 2) % 8 != 0) {
        std::fprintf(stderr, "usage: %s G (slot nbx nby nbz bsx bsy bsz ntile)...\n", argv[0]);
        return 2;
    }
    const long long G = std::atoll(argv[1]);
    std::vector<orcha::ColumnSource> src;
    for (int a = 2; a + 7 < argc; a += 8) {
        orcha::ColumnSource c;
        c.slot = std::atoi(argv[a]);
        for (int d = 0; d < 3; ++d) {
            c.nb[d] = std::atoi(argv[a + 1 + d]);
            c.bs[d] = std::atoi(argv[a + 4 + d]);
        }
        c.ntile = std::atoi(argv[a + 7]);
        src.push_back(c);
    }
    for (const orcha::Item& it : orcha::column_items(src, G))
        std::printf("%d %d %d %d %d\n", it.slot, it.blk, it.tile, it.zr & 0xFFFF, it.zr >> 16);
    return 0;
}
