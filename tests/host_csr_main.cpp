// Test driver for the library's host CSR build (no GPU): reads n, m and the
// arc arrays from a binary file, builds the dual CSR and writes it back.
//   in : int64 n, int64 m, int32 src[m], int32 dst[m]
//   out: int64 status, int64 arcs, int32 out_off[n+1], out_adj[arcs],
//        int32 in_off[n+1], in_adj[arcs]
// Several inputs may follow each other in one file; each gets a build in
// turn (the build keeps its staging arrays between calls).
#include <cstdio>
#include <string>
#include <vector>

#include "xm_internal.h"

void xm::set_error(const std::string&) {}

int main(int argc, char** argv) {
    if (argc != 3) return 2;
    FILE* in = fopen(argv[1], "rb");
    FILE* out = fopen(argv[2], "wb");
    if (!in || !out) return 2;
    xm::HostCsr G;
    int64_t hdr[2];
    while (fread(hdr, sizeof(int64_t), 2, in) == 2) {
        const int64_t n = hdr[0], m = hdr[1];
        std::vector<int32_t> s((size_t)m), d((size_t)m);
        if (m && (fread(s.data(), 4, (size_t)m, in) != (size_t)m || fread(d.data(), 4, (size_t)m, in) != (size_t)m))
            return 2;
        std::string err;
        const int64_t rc = xm::build_host_csr((int32_t)n, m, s.data(), d.data(), G, err);
        const int64_t arcs = rc ? 0 : G.m;
        fwrite(&rc, 8, 1, out);
        fwrite(&arcs, 8, 1, out);
        if (rc) continue;
        fwrite(G.out_off.data(), 4, (size_t)n + 1, out);
        fwrite(G.out_adj.data(), 4, (size_t)arcs, out);
        fwrite(G.in_off.data(), 4, (size_t)n + 1, out);
        fwrite(G.in_adj.data(), 4, (size_t)arcs, out);
    }
    fclose(out);
    return 0;
}
