// The paper's decomposition of the transform over several GPUs (Sec. 3.1.1):
// every rank owns a set of zonal wavenumbers m, for which it runs the
// Legendre transform over all latitudes, and a set of latitude ring pairs,
// for which it runs the ring FFTs.  Between the two, every rank exchanges
// the Fourier coefficients with every other rank once per direction (the
// all-to-all of Sec. 3.1.1 and Sec. 3.1.3.2), with the packing and unpacking
// on the device (Sec. 3.1.3.1):
//   inverse  Legendre (own m, all rings) -> pack per destination rank the rows
//            (its rings, own m) -> all-to-all -> unpack (own rings, every m)
//            -> ring FFTs (own rings)
//   direct   ring FFTs (own rings, every m) -> pack per destination rank the
//            rows (its m, own rings) -> all-to-all -> unpack (own m, every
//            ring) -> Legendre (own m)
// The library provides the partitioned plan, the four half-transforms and
// the pack/unpack kernels; the exchange itself is the caller's collective
// (NCCL's all-to-all in the Python driver, gloo in the host tests).  The row
// lists of the exchange are built here, once, when the partition is set, so
// the transform calls still allocate nothing.
#include <string.h>

#include <algorithm>

#include "st_internal.cuh"

namespace st {

void part_free(Plan* p)
{
    if (!p->part) return;
    for (int d = 0; d < 2; d++) {
        if (p->part->d_send[d]) cudaFree(p->part->d_send[d]);
        if (p->part->d_recv[d]) cudaFree(p->part->d_recv[d]);
    }
    if (p->part->d_mown) cudaFree(p->part->d_mown);
    delete p->part;
    p->part = nullptr;
}

namespace {

// the northern ring pair of ring k (0 .. nlat-1)
inline int pair_of(const Tables* t, int k) { return k < t->N ? k : t->nlat - 1 - k; }

// rows of direction d that the sender `from` ships to the receiver `to`, in
// the order both sides enumerate them
void exchange_rows(const Tables* t, const PartInfo& q, int d, int from, int to, std::vector<long>& rows)
{
    if (d == 0) {  // inverse: Fourier rows (ring k of `to`, m of `from`)
        for (int k = 0; k < t->nlat; k++) {
            if (q.ring_owner[pair_of(t, k)] != to) continue;
            for (int m = 0; m <= t->mmax[k]; m++)
                if (q.m_owner[m] == from) rows.push_back(t->foff[k] + m);
        }
    } else {  // direct: operand rows (m of `to`, both parities, ring pair of `from`)
        for (int m = 0; m <= t->T; m++) {
            if (q.m_owner[m] != to) continue;
            for (int par = 0; par < 2; par++)
                for (int l = 0; l < t->L[m]; l++)
                    if (q.ring_owner[t->k0[m] + l] == from) rows.push_back(t->goff[2 * m + par] + l);
        }
    }
}

// copy nrows rows of ncols elements (4 or 8 bytes): pack gathers rows[i] of
// the strided array into row i of the contiguous buffer; unpack scatters back
template <typename E>
__global__ void k_rows_copy(E* __restrict__ arr, E* __restrict__ buf, const long* __restrict__ rows, long nrows,
                            int ncols, long stride, int pack)
{
    const long n = nrows * (long)ncols;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const long r = i / ncols;
        const int c = (int)(i - r * ncols);
        E* a = arr + rows[r] * stride + c;
        if (pack) buf[i] = *a;
        else *a = buf[i];
    }
}

// the array a direction exchanges, and its element size
void* exchange_array(const Plan* p, int d, int* eb)
{
    const bool f64 = p->opts.prec == ST_PREC_FP64;
    *eb = f64 ? 8 : 4;
    if (d == 1 && p->ws_gop32) return p->ws_gop32;  // split paths: the FP32 direct operand
    return p->ws_four;
}

}  // namespace

}  // namespace st

using namespace st;

extern "C" {

int st_plan_set_partition(st_plan* pp, int nranks, int rank, const int* m_owner, const int* ring_owner)
{
    if (!pp || nranks < 1 || rank < 0 || rank >= nranks || !m_owner || !ring_owner) {
        set_error("st_plan_set_partition: bad argument");
        return ST_ERR_ARG;
    }
    Plan* p = (Plan*)pp;
    const Tables* t = p->tab;
    for (int m = 0; m <= p->T; m++)
        if (m_owner[m] < 0 || m_owner[m] >= nranks) {
            set_error("st_plan_set_partition: m_owner[%d] = %d outside [0, %d)", m, m_owner[m], nranks);
            return ST_ERR_ARG;
        }
    for (int k = 0; k < t->N; k++)
        if (ring_owner[k] < 0 || ring_owner[k] >= nranks) {
            set_error("st_plan_set_partition: ring_owner[%d] = %d outside [0, %d)", k, ring_owner[k], nranks);
            return ST_ERR_ARG;
        }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_error("st_plan_set_partition: %s", cudaGetErrorString(cudaGetLastError()));
        return ST_ERR_CUDA;
    }
    PartInfo* q = new PartInfo();
    q->nranks = nranks;
    q->rank = rank;
    q->m_owner.assign(m_owner, m_owner + p->T + 1);
    q->ring_owner.assign(ring_owner, ring_owner + t->N);
    int rc = ST_OK;
    for (int d = 0; d < 2 && rc == ST_OK; d++) {
        std::vector<long> send, recv;
        for (int r = 0; r < nranks; r++) {
            size_t s0 = send.size(), r0 = recv.size();
            exchange_rows(t, *q, d, rank, r, send);
            exchange_rows(t, *q, d, r, rank, recv);
            q->send_cnt[d].push_back((long)(send.size() - s0));
            q->recv_cnt[d].push_back((long)(recv.size() - r0));
        }
        q->nsend[d] = (long)send.size();
        q->nrecv[d] = (long)recv.size();
        if (dev_malloc((void**)&q->d_send[d], std::max<size_t>(send.size(), 1) * sizeof(long)) != cudaSuccess ||
            dev_malloc((void**)&q->d_recv[d], std::max<size_t>(recv.size(), 1) * sizeof(long)) != cudaSuccess) {
            cudaGetLastError();
            rc = ST_ERR_NOMEM;
            break;
        }
        if ((!send.empty() && cudaMemcpy(q->d_send[d], send.data(), send.size() * sizeof(long), cudaMemcpyHostToDevice) !=
                                  cudaSuccess) ||
            (!recv.empty() && cudaMemcpy(q->d_recv[d], recv.data(), recv.size() * sizeof(long), cudaMemcpyHostToDevice) !=
                                  cudaSuccess))
            rc = ST_ERR_CUDA;
    }
    if (rc == ST_OK) {  // the owned wavenumbers, for the kernels that run over all m
        std::vector<unsigned char> own(p->T + 1);
        for (int m = 0; m <= p->T; m++) own[m] = m_owner[m] == rank;
        if (dev_malloc((void**)&q->d_mown, own.size()) != cudaSuccess) {
            cudaGetLastError();
            rc = ST_ERR_NOMEM;
        } else if (cudaMemcpy(q->d_mown, own.data(), own.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
            rc = ST_ERR_CUDA;
        }
    }
    if (rc != ST_OK) {  // the plan keeps its previous partition
        Plan tmp;
        memset((void*)&tmp, 0, sizeof tmp);
        tmp.part = q;
        part_free(&tmp);
        set_error("st_plan_set_partition: %s", rc == ST_ERR_NOMEM ? "out of device memory" : "row lists");
        return rc;
    }
    // swap in the new partition and the work lists it restricts
    PartInfo* old = p->part;
    p->part = q;
    free_leg_worklists(p);
    if (p->d_spec_chunks) cudaFree(p->d_spec_chunks);
    if (p->d_fft_items) cudaFree(p->d_fft_items);
    if (p->d_fft_ctas) cudaFree(p->d_fft_ctas);
    p->d_spec_chunks = nullptr;
    p->d_fft_items = p->d_fft_ctas = nullptr;
    rc = build_leg_worklists(p);
    if (old) {
        Plan tmp;
        memset((void*)&tmp, 0, sizeof tmp);
        tmp.part = old;
        part_free(&tmp);
    }
    if (rc != ST_OK) {
        set_error("st_plan_set_partition: %s", rc == ST_ERR_NOMEM ? "out of device memory" : "work lists");
        return rc;
    }
    return ST_OK;
}

int st_exchange_counts(const st_plan* pp, int dir, long* send_rows, long* recv_rows, int* row_bytes)
{
    if (!pp || (dir != 0 && dir != 1)) {
        set_error("st_exchange_counts: bad argument");
        return ST_ERR_ARG;
    }
    const Plan* p = (const Plan*)pp;
    if (!p->part) {
        set_error("st_exchange_counts: the plan has no partition");
        return ST_ERR_ARG;
    }
    int eb = 0;
    exchange_array(p, dir, &eb);
    if (row_bytes) *row_bytes = 2 * p->nfld * eb;
    for (int r = 0; r < p->part->nranks; r++) {
        if (send_rows) send_rows[r] = p->part->send_cnt[dir][r];
        if (recv_rows) recv_rows[r] = p->part->recv_cnt[dir][r];
    }
    return ST_OK;
}

static int exchange_copy(st_plan* pp, int dir, void* buf, void* stream, bool pack, const char* fn)
{
    if (!pp || !buf || (dir != 0 && dir != 1)) {
        set_error("%s: bad argument", fn);
        return ST_ERR_ARG;
    }
    Plan* p = (Plan*)pp;
    if (!p->part) {
        set_error("%s: the plan has no partition", fn);
        return ST_ERR_ARG;
    }
    int eb = 0;
    void* arr = exchange_array(p, dir, &eb);
    const long nrows = pack ? p->part->nsend[dir] : p->part->nrecv[dir];
    const long* rows = pack ? p->part->d_send[dir] : p->part->d_recv[dir];
    if (nrows == 0) return ST_OK;
    const int ncols = 2 * p->nfld;
    const long n = nrows * ncols;
    const int nb = (int)std::min<long>((n + 255) / 256, 152L * 16);
    cudaStream_t s = (cudaStream_t)stream;
    if (eb == 8) k_rows_copy<double><<<nb, 256, 0, s>>>((double*)arr, (double*)buf, rows, nrows, ncols, p->ncolp, pack);
    else k_rows_copy<float><<<nb, 256, 0, s>>>((float*)arr, (float*)buf, rows, nrows, ncols, p->ncolp, pack);
    ST_CUDA_TRY(cudaGetLastError());
    p->last_launches = 1;
    return ST_OK;
}

int st_exchange_pack(st_plan* p, int dir, void* buf, void* stream)
{
    return exchange_copy(p, dir, buf, stream, true, "st_exchange_pack");
}

int st_exchange_unpack(st_plan* p, int dir, const void* buf, void* stream)
{
    return exchange_copy(p, dir, const_cast<void*>(buf), stream, false, "st_exchange_unpack");
}

}  // extern "C"
