// Internal definitions shared by the host and device translation units of
// libbpq.  Not part of the public ABI (include/bpq.h is).
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/bpq.h"

namespace bpq {

constexpr int kMaxDeg = 4;          // padded check and qubit degree of the decoder
constexpr int kMaxThreadsPerShot = 1024;
constexpr int kMaxNodesPerThread = 4;
constexpr int kMaxNodes = 2048;  // max(N, M): two nodes per thread at 1024 threads per shot
constexpr uint16_t kNoSlot = 0xFFFF;
constexpr size_t kWorkspaceBytes = 256;  // [0] next shot, [1] device error word

void set_error(const std::string &msg);
int fail(int code, const std::string &msg);

}  // namespace bpq

// Tanner graph handle.  Host fields are filled by the builders; device
// fields by bpq_tanner_upload.
struct bpq_tanner {
    int N = 0, M = 0, E = 0, K = -1;
    int code = -1, d = 0;
    // check-major CSR, neighbours in increasing qubit order
    std::vector<int32_t> chk_ptr, chk_var;
    std::vector<uint8_t> chk_pauli;
    std::vector<uint8_t> logicals;  // 2K x N Pauli codes (empty if unknown)

    // Decoder adjacency tables (built by bpq::build_tables), generic layout:
    //  slot of edge (qubit j, k-th check of j in increasing check order)
    //  = 4 j + ((k + j / 8) mod 4)
    std::vector<uint8_t> table;      // [chk_slot u16 M_pad x 4][chk_pauli u8 M_pad][var_pauli u8 N_pad]
    uint32_t off_chk_pauli = 0, off_var_pauli = 0;
    std::vector<int32_t> var_canon;  // 4N: check-major edge index of each slot (-1 = padding)
    // Split layout, for codes without Y entries whose qubits have at most two
    // X edges and two Z edges (every surface code here): the same table
    // format, but slot p * n4 + j (n4 = N rounded up to 4) holds qubit j's
    // p-th edge with positions 0, 1 its X edges and 2, 3 its Z edges.
    bool split = false;
    std::vector<uint8_t> table_split;
    std::vector<int32_t> var_canon_split;  // 4 n4, indexed by split slot

    // device
    int device = -1;
    void *dev_blob = nullptr;
    const uint8_t *d_table = nullptr;
    const int32_t *d_var_canon = nullptr;
    const uint8_t *d_table_split = nullptr;
    const int32_t *d_var_canon_split = nullptr;
    const int32_t *d_chk_ptr = nullptr;
    const uint8_t *d_logicals = nullptr;
    int num_sms = 0;

    // launch preferences (0 = automatic)
    int threads_per_shot = 0, shots_per_cta = 0;
};

namespace bpq {
// Fill t->table, offsets and var_canon from the CSR; returns BPQ_OK or an error.
int build_tables(bpq_tanner *t);
}  // namespace bpq
