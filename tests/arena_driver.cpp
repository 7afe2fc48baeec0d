// Command-line driver for the render server's arena allocator (host C++):
// reads "init S", "alloc B", "release OFF B" and "state" lines on stdin
// and prints each result, for tests/test_arena.py to compare with a model.
#include <cstdio>
#include <cstring>

#include "arena.h"

int main() {
    msgs::Arena a;
    char op[16];
    while (std::scanf("%15s", op) == 1) {
        unsigned long long x = 0, y = 0;
        if (!std::strcmp(op, "init") && std::scanf("%llu", &x) == 1) {
            a.init((size_t)x);
            std::printf("ok\n");
        } else if (!std::strcmp(op, "alloc") && std::scanf("%llu", &x) == 1) {
            size_t off = 0;
            if (a.alloc((size_t)x, off)) std::printf("ok %llu\n", (unsigned long long)off);
            else std::printf("fail\n");
        } else if (!std::strcmp(op, "release") && std::scanf("%llu %llu", &x, &y) == 2) {
            a.release((size_t)x, (size_t)y);
            std::printf("ok\n");
        } else if (!std::strcmp(op, "state")) {
            std::printf("%llu %llu %llu", (unsigned long long)a.size(),
                        (unsigned long long)a.used(), (unsigned long long)a.peak());
            for (const auto &r : a.free_ranges())
                std::printf(" %llu:%llu", (unsigned long long)r.first,
                            (unsigned long long)r.second);
            std::printf("\n");
        } else {
            std::printf("bad\n");
            return 1;
        }
    }
    return 0;
}
