// Test helper (host only, no GPU): lowers one protocol, packs it with the
// range pass planned whatever its size, and writes the sort-path keys of its
// range pieces -- k0 + o * d for each piece's threads o -- so that a CPU test
// can compare them with the oracle's accesses.
//
//   range_keys_dump OUT NTHREADS BYTECODE_HEX CELLS...
//
// OUT: 8 little-endian uint64 (proto, phase, loc, index and tid bits of the
// key layout, the protocol's access instructions, those of them in the range
// pass, the number of keys), then the keys.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "host/engine.h"
#include "host/prepare.h"

using namespace drf;

int main(int argc, char **argv)
{
    if (argc < 4) {
        std::fprintf(stderr, "usage: %s OUT NTHREADS BYTECODE_HEX CELLS...\n", argv[0]);
        return 2;
    }
    const uint32_t nthreads = (uint32_t)std::strtoul(argv[2], nullptr, 10);
    const std::string hex = argv[3];
    std::vector<uint8_t> bc(hex.size() / 2);
    for (size_t i = 0; i < bc.size(); i++) bc[i] = (uint8_t)std::stoul(hex.substr(2 * i, 2), nullptr, 16);
    std::vector<uint64_t> cells;
    for (int i = 4; i < argc; i++) cells.push_back(std::strtoull(argv[i], nullptr, 10));
    Prepared p;
    PrepareOpts po;
    Error e = prepare(bc.data(), bc.size(), nthreads, (uint32_t)cells.size(), cells.data(), 0, nullptr, po, p);
    if (!e.ok()) {
        std::fprintf(stderr, "prepare: %s\n", e.message.c_str());
        return 1;
    }
    BatchHost bh;
    e = pack_batch({&p}, bh, true, 0, 0);
    if (!e.ok()) {
        std::fprintf(stderr, "pack: %s\n", e.message.c_str());
        return 1;
    }
    uint64_t acc = 0, racc = 0;
    for (const Insn &in : bh.insns)
        if (in.op == I_ACCESS || in.op == I_FASTACC) {
            acc++;
            racc += (in.a & AF_RANGE) ? 1 : 0;
        }
    std::vector<uint64_t> out = {bh.L.proto_bits, bh.L.phase_bits, bh.L.loc_bits, bh.L.idx_bits, bh.L.tid_bits,
                                 acc, racc, bh.nrkeys};
    for (const RKeys &k : bh.wkeys) {
        if (k.pre != out.size() - 8) {
            std::fprintf(stderr, "piece keys out of order\n");
            return 1;
        }
        for (uint64_t o = 0; o < k.len; o++) out.push_back(k.k0 + o * k.d);
    }
    if (out.size() - 8 != bh.nrkeys) {
        std::fprintf(stderr, "key count mismatch\n");
        return 1;
    }
    FILE *f = std::fopen(argv[1], "wb");
    if (!f || std::fwrite(out.data(), 8, out.size(), f) != out.size()) return 1;
    std::fclose(f);
    return 0;
}
