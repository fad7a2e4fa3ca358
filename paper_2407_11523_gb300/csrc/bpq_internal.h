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

// Alignment the entry points require of caller buffers: device buffers passed
// as void * (workspaces, the host path's buffer, a server's device memory) are
// cut into 32-bit words and descriptors with 64-bit fields, which kernels may
// copy in 16-byte bulk copies; syndromes and priors are read as 32-bit words.
// A base off these boundaries would make the device accesses misaligned, so
// the entry points refuse it (BPQ_EINVAL) instead.
constexpr size_t kBufferAlign = 16, kWordAlign = 4;
inline bool misaligned(const void *p, size_t align) {
    return (reinterpret_cast<uintptr_t>(p) & (align - 1)) != 0;
}

// One qubit of the serial schedule's sweep (48 bytes, 16-byte aligned); the
// serial table lists them level by level (see serial.cu).  Message slots
// index the kernel's per-shot message array: every edge has one slot, laid
// out so that the lanes of one access fall in distinct shared-memory banks;
// two extra slots follow the edges' (zero: reads as a certain message with
// positive sign, the identity of the check rule; trash: takes writes of
// padding edges).
struct SerialVar {
    uint16_t own[4];     // slot of the qubit's edge k (the trash slot for padding)
    uint16_t oth[4][3];  // slots of the other edges of edge k's check (the zero slot for padding)
    uint16_t chk[4];     // the check of edge k (0 for padding)
    uint16_t j;          // the qubit
    uint8_t pauli;       // H_ij of edge k in bits 2k, 2k+1 (0 for padding)
    uint8_t last;        // bit k: the qubit is the last of edge k's check in the sweep
    uint8_t real;        // bit k: edge k exists (not padding)
    uint8_t pad[3];
};
static_assert(sizeof(SerialVar) == 48, "SerialVar layout");

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
    // Split layout with every slot in use: every check has four edges and
    // every qubit two X and two Z edges (the toric codes), so the decoder
    // needs no padding slots.
    bool full = false;
    std::vector<uint8_t> table_split;
    std::vector<int32_t> var_canon_split;  // 4 n4, indexed by split slot
    // Serial schedule (bpq::build_serial_table): SerialVar[N] in level order |
    // level_ptr u16[levels + 1] | canon u16[N][4] (check-major index of each
    // qubit's edge k, E for padding; 16-byte aligned, read by the trace
    // kernels only, so the kernels stage the table up to it), padded to 16
    // bytes; serial_slots
    // message slots for the edges, then the zero and the trash slot.
    std::vector<uint8_t> serial;
    int serial_levels = 0, serial_slots = 0;
    uint32_t serial_off_levels = 0, serial_off_canon = 0;

    // device
    int device = -1;
    void *dev_blob = nullptr;
    const uint8_t *d_table = nullptr;
    const int32_t *d_var_canon = nullptr;
    const uint8_t *d_table_split = nullptr;
    const uint8_t *d_serial = nullptr;
    const int32_t *d_var_canon_split = nullptr;
    const int32_t *d_chk_ptr = nullptr;
    const uint8_t *d_logicals = nullptr;
    int num_sms = 0;

    // launch preferences (0 = automatic); with two shots per thread the
    // first two describe a shot group (which decodes two shots at a time)
    int threads_per_shot = 0, shots_per_cta = 0, shots_per_thread = 0;
    // nodes per thread inside the batched kernel and the servers (0 = automatic)
    int batch_nodes_per_thread = 0;
    // shots per warp of the serial-schedule kernel (0 = automatic)
    int serial_shots_per_warp = 0;
    // run the bounds-checked kernels (bpq_set_debug_checks)
    bool debug_checks = false;
};

namespace bpq {
// Fill t->table, offsets and var_canon from the CSR; returns BPQ_OK or an error.
int build_tables(bpq_tanner *t);
// Fill t->serial (called by build_tables).
int build_serial_table(bpq_tanner *t);
}  // namespace bpq
