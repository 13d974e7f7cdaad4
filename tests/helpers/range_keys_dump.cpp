// Test helper (host only, no GPU): lowers one protocol, packs it with the
// range pass planned whatever its size, and writes what the range pass was
// planned to do, so that a CPU test can compare it with the oracle's
// accesses.
//
//   range_keys_dump [--pieces] OUT NTHREADS BYTECODE_HEX CELLS...
//
// Keys (default): 9 little-endian uint64 (proto, phase, loc, index and tid
// bits of the key layout, the protocol's access instructions, those of them
// in the range pass, the access tuples those make as counted on the host,
// the number of keys), then the sort-path keys of the range pieces,
// k0 + o * d for each piece's threads o.
//
// --pieces: uint64 header (records per task, tab_off, cells_sum, tab_phases,
// nlocs, the number of task entries, of merged pieces, the access
// instructions and those in the range pass), the nlocs array offsets within a
// phase row (cbase), then the task entries (task, p0, p1, win: 4 uint32 each)
// and the merged pieces (t0, lenf, l0, step: 4 x 32 bits each), as the range
// kernel receives them.
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
    const bool pieces = argc > 1 && std::string(argv[1]) == "--pieces";
    if (pieces) {
        argv++;
        argc--;
    }
    if (argc < 4) {
        std::fprintf(stderr, "usage: %s [--pieces] OUT NTHREADS BYTECODE_HEX CELLS...\n", argv[0]);
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
    if (pieces) {
        const DevProto &d = bh.protos.at(0);
        std::vector<uint64_t> hdr = {kRangeRecs, d.tab_off, d.cells_sum, d.tab_phases, d.nlocs,
                                     bh.rtask.size(), bh.rpiece.size(), acc, racc};
        for (uint32_t l = 0; l < d.nlocs; l++) hdr.push_back(bh.cbase[d.cells_off + l]);
        FILE *f = std::fopen(argv[1], "wb");
        bool ok = f && std::fwrite(hdr.data(), 8, hdr.size(), f) == hdr.size();
        ok = ok && (bh.rtask.empty() || std::fwrite(bh.rtask.data(), sizeof(RTask), bh.rtask.size(), f) == bh.rtask.size());
        ok = ok && (bh.rpiece.empty() ||
                    std::fwrite(bh.rpiece.data(), sizeof(RPiece), bh.rpiece.size(), f) == bh.rpiece.size());
        if (f) std::fclose(f);
        return ok ? 0 : 1;
    }
    std::vector<uint64_t> out = {bh.L.proto_bits, bh.L.phase_bits, bh.L.loc_bits, bh.L.idx_bits, bh.L.tid_bits,
                                 acc, racc, bh.range_tuples, bh.nrkeys};
    const size_t hdr = out.size();
    for (const RKeys &k : bh.wkeys) {
        if (k.pre != out.size() - hdr) {
            std::fprintf(stderr, "piece keys out of order\n");
            return 1;
        }
        for (uint64_t o = 0; o < k.len; o++) out.push_back(k.k0 + o * k.d);
    }
    if (out.size() - hdr != bh.nrkeys) {
        std::fprintf(stderr, "key count mismatch\n");
        return 1;
    }
    FILE *f = std::fopen(argv[1], "wb");
    if (!f || std::fwrite(out.data(), 8, out.size(), f) != out.size()) return 1;
    std::fclose(f);
    return 0;
}
