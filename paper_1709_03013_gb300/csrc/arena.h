// One device allocation holding a launch sequence's tables and scratch.
//
// Host code builds the tables into an image (put), reserves device-only scratch
// (reserve), allocates once, patches address-dependent entries into the image,
// uploads the image with a single copy, and then enqueues kernels that read the
// tables and use the scratch.  Nothing in the enqueue step allocates or
// synchronises, so the same sequence can be captured into a CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <string.h>

#include <vector>

namespace csg {

struct Arena {
    static constexpr size_t kAlign = 256;
    std::vector<unsigned char> img;  // table image (uploaded)
    size_t scratch_bytes = 0;        // device-only region after the tables
    unsigned char *dev = nullptr;

    static size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
    size_t table_bytes() const { return up(img.size()); }
    size_t bytes() const { return table_bytes() + scratch_bytes; }

    // Appends n bytes (copied from p when non-null, else zeroed) to the table image.
    size_t put(const void *p, size_t n) {
        const size_t off = up(img.size());
        img.resize(off + (n ? n : 1), 0);
        if (p && n) memcpy(&img[off], p, n);
        return off;
    }
    template <typename T>
    T *host(size_t off) {
        return reinterpret_cast<T *>(&img[off]);
    }
    // Reserves n bytes of device-only scratch.
    size_t reserve(size_t n) {
        const size_t off = up(scratch_bytes);
        scratch_bytes = off + (n ? n : 1);
        return off;
    }
    template <typename T>
    T *tab(size_t off) const {
        return reinterpret_cast<T *>(dev + off);
    }
    template <typename T>
    T *scr(size_t off) const {
        return reinterpret_cast<T *>(dev + table_bytes() + off);
    }
    // Device address a scratch offset will have (valid once dev is set).
    template <typename T>
    T *scr_addr(size_t off) const {
        return scr<T>(off);
    }
};

}  // namespace csg
