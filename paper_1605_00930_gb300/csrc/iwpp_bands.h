// iwpp_bands.h — the visit order of the out-of-core reconstruction's bands (host logic only,
// no CUDA: iwpp_ooc.cu drives it, and a host test drives it against a simulated image).
//
// Every band is visited once; after that a band is visited again only when a neighbour band
// changed after its last visit (its overlap and halo rows may then differ). Visits sweep top to bottom,
// then bottom to top, skipping clean bands, until no band is dirty. When next() returns -1,
// every band's last visit saw its neighbours' final rows.
#pragma once

#include <cstdint>
#include <vector>

namespace iwpp {

// Rows of each neighbour band reconstructed together with a band of `band` rows and not
// written back (the overlap; always < band, so an extended band reaches only its two
// neighbours).
inline int64_t band_overlap(int64_t band) { return band / 16; }

class BandSchedule {
  public:
    explicit BandSchedule(int64_t nbands) : dirty_((size_t)(nbands > 0 ? nbands : 0), 1), ndirty_(nbands > 0 ? nbands : 0) {}

    // The next band to visit, or -1 when none is dirty.
    int64_t next() {
        const int64_t nb = (int64_t)dirty_.size();
        while (ndirty_ > 0) {
            for (; pos_ < nb; pos_++) {
                const int64_t b = down_ ? pos_ : nb - 1 - pos_;
                if (dirty_[(size_t)b]) {
                    pos_++;
                    return b;
                }
            }
            pos_ = 0;
            down_ = !down_;
        }
        return -1;
    }

    // The band next() would return after visited(b, true): the best guess of the next visit
    // while band b is still being reconstructed (a band that changes dirties its neighbours).
    int64_t peek_after_change(int64_t b) const {
        BandSchedule t = *this;
        t.visited(b, true);
        return t.next();
    }

    // Report the visit of band b: it is clean now; if its rows changed, its neighbours are dirty.
    void visited(int64_t b, bool changed) {
        const int64_t nb = (int64_t)dirty_.size();
        if (b < 0 || b >= nb) return;
        if (dirty_[(size_t)b]) {
            dirty_[(size_t)b] = 0;
            ndirty_--;
        }
        if (!changed) return;
        for (int64_t n : {b - 1, b + 1})
            if (n >= 0 && n < nb && !dirty_[(size_t)n]) {
                dirty_[(size_t)n] = 1;
                ndirty_++;
            }
    }

  private:
    std::vector<char> dirty_;
    int64_t ndirty_;
    int64_t pos_ = 0;
    bool down_ = true;
};

}  // namespace iwpp
