// kernels.h -- launch interface of the device kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include "plan.h"

namespace ata {

// Device pointers an execution binds: the caller's A (X of a general
// product), Y (general product only) and C, and the plan's workspace, per
// instance.  Kernels receive a BindSet by value (a __grid_constant__
// parameter), so a launch snapshots its pointers and a captured graph is
// re-pointed by updating kernel-node parameters.
struct Bind {
    const void* A;
    double* C;
    char* W;
    int64_t n;
    // extents for the optional self-check of every global access (check != 0):
    // elements of A, bytes of W, elements of C
    int64_t a_elems, w_bytes, c_elems;
    int64_t check;
    const void* B;
    int64_t b_elems;
};

// Base of the buffer a term reads (A, Y of a general product, or W).
template <typename T>
__host__ __device__ __forceinline__ const T* term_base(const Bind& b, int8_t buf) {
    return reinterpret_cast<const T*>(buf == BUF_A ? b.A : buf == BUF_B ? b.B : static_cast<const void*>(b.W));
}

// Bindings of a launch: one instance by value (NB == 1, in the kernel's
// parameter space), or any number read from a device array (NB == kDevBinds,
// batched launches; the array is filled before the launch).  Kernels index
// bs.b[inst] either way.
constexpr int kDevBinds = 0;

template <int NB>
struct BindSet {
    Bind b[NB];
};

template <>
struct BindSet<kDevBinds> {
    const Bind* b;
};

// One output tile of the leaf launch, or one K range of it (FP64 leaves cut
// along K: part >= 0 is the partial tile's slot in the product's region).
struct LeafTile {
    int32_t prod;
    int32_t ti, tj;
    int32_t k0, k1;           // K range [k0, k1)
    int32_t part;             // -1: the whole K, output written directly
};

// Sum of one cut tile's partials, in part order, into its output.
struct PartialSum {
    int32_t prod;
    int32_t ti, tj;
    int32_t slot0;            // first partial slot (kparts of them)
};

// A range of rows of an elementwise task (split or combine).
struct Chunk {
    int32_t task;
    int32_t row0, nrows;
};

constexpr int kMaxTerms = 32;     // terms per operand the leaf kernels accept

// `binds`: nb == 1, the one instance in host memory (passed by value, the
// single-plan instantiation of each kernel); nb > 1, a device array of nb
// instances (the kDevBinds instantiation).
// `status` receives a nonzero code when a self-checked access falls outside its
// buffer (the access is skipped): 11 leaf read, 12 leaf write, 21 split read,
// 22 split write, 31 combine read, 32 combine write.
// Partials of FP64 tiles cut along K, added in part order into the outputs.
cudaError_t launch_partial_sums(int* status, const Bind* binds, int nb, const LeafProduct* prods,
                                const PartialSum* tasks, int ntasks, cudaStream_t s);
cudaError_t launch_leaf_f64(int* status, const Bind* binds, int nb, const LeafProduct* prods, const Term* terms, const LeafTile* tiles,
                            int ntiles, int* counter, int grid, cudaStream_t s);

cudaError_t launch_split(int* status, const Bind* binds, int nb, const SplitTask* tasks, const Chunk* chunks, int nchunks, int8_t src_dt,
                         int8_t dst_dt, cudaStream_t s);

cudaError_t launch_combine(int* status, const Bind* binds, int nb, const CombineTask* tasks, const Chunk* chunks, int nchunks,
                           cudaStream_t s);

// Resident blocks of the FP64 leaf kernel per SM (for persistent grids).
int leaf_f64_blocks_per_sm();

}  // namespace ata
