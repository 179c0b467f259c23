// Domain-decomposed Wilson-Clover operator with the halo exchange overlapped
// by computation (Sec. 2.2: the paper splits its multi-node hopping
// multiplication into a pre-communication step, an interior step that runs
// while the messages travel, and a post-communication step for the surface).
//
// A sub-domain (wc_create_subdomain) is a lattice holding the sites
// [offset, offset + L) of a larger lattice; a direction is cut when the
// sub-domain is shorter than the whole lattice along it.  The operator of a
// sub-domain is applied in three launches:
//
//   wc_halo_pack      (pre)  the face data the neighbours need, 12 reals per
//                            face site (a colour two-spinor pair):
//                            to the lower neighbour  h = (1 + s_f g_mu) psi(y)
//                            at the lower-face sites y (the receiver applies
//                            its own link U_mu(x), x = y - mu);
//                            to the upper neighbour  w = U_mu(y)^+ (1 + s_b g_mu)
//                            psi(y) at the upper-face sites y (the link lives
//                            with the sender);
//   wc_apply_interior (in)   every site without a hop across a cut face --
//                            the same per-site code as the whole-lattice
//                            kernel, so these sites are bit-identical to it;
//   wc_apply_surface  (post) the remaining sites, taking the hops across cut
//                            faces from the received buffers in the same
//                            arithmetic order as the whole-lattice kernel
//                            (the received h and w are exactly the values
//                            that kernel forms from the neighbour spinor).
//
// s_f = -1, s_b = +1 for M; M^+ swaps them.  The time-boundary factor of a
// hop across a cut t face applies when the hop crosses the global time
// boundary.  FP32 storage and arithmetic (the paper's single-precision
// MULT).  Buffers are float4 planes [3][nface] (a face site's six complex
// values), face sites ordered lexicographically in the three other
// directions (x fastest); the sender and receiver agree on this order
// because neighbouring sub-domains have the same extents across the face.
//
// The gauge field of a sub-domain is loaded with a one-site halo across
// every cut face: the clover leaves of a face site reach one site into the
// neighbours.  The extended field lives in an internal lattice on which the
// clover term is built; its interior is copied into the sub-domain.
#include "wc_internal.cuh"
#include "wc_stencil.cuh"

namespace wc {

namespace {

constexpr int kHaloThreads = 128;

struct HaloGeom {
    int split_mask;
    int nface[4];         // V / L[mu]
    int fwd_cross_t;      // the upper t face borders the global time boundary
    int bwd_cross_t;      // the lower t face borders it
};

struct HaloBufs {
    const float4 *from_lower[4];   // w values of the lower neighbour's upper face
    const float4 *from_upper[4];   // h values of the upper neighbour's lower face
};

// face index of site coordinates c on a face normal to mu
template <int MU>
__device__ __forceinline__ int face_index(const Geom &g, const int c[4])
{
    int f = 0, s = 1;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (m == MU) continue;
        f += c[m] * s;
        s *= g.L[m];
    }
    return f;
}

// coordinates of face site f on the face c[MU] = cm
template <int MU>
__device__ __forceinline__ int face_site(const Geom &g, int f, int cm, int c[4])
{
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        if (m == MU) {
            c[m] = cm;
            continue;
        }
        c[m] = f % g.L[m];
        f /= g.L[m];
    }
    return c[0] + g.stride[1] * c[1] + g.stride[2] * c[2] + g.stride[3] * c[3];
}

__device__ __forceinline__ void store6(float4 *buf, int n, int f, const cx<float> v[6])
{
#pragma unroll
    for (int j = 0; j < 3; ++j) buf[(size_t)j * n + f] = make_float4(v[2 * j].re, v[2 * j].im, v[2 * j + 1].re, v[2 * j + 1].im);
}

__device__ __forceinline__ void load6(const float4 *buf, int n, int f, cx<float> v[6])
{
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float4 t = __ldg(buf + (size_t)j * n + f);
        v[2 * j] = mkc(t.x, t.y);
        v[2 * j + 1] = mkc(t.z, t.w);
    }
}

// pre: the two face buffers of direction MU
template <int MU, int SF>
__global__ void __launch_bounds__(kHaloThreads) k_halo_pack(Geom g, int nface, GaugeStore U, const void *in,
                                                            float4 *to_lower, float4 *to_upper)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nface) return;
    constexpr int SB = -SF;
    int c[4];
    {
        const int y = face_site<MU>(g, f, 0, c);
        cx<float> p[12], h[6];
        P32::load_spinor(in, nullptr, g.V, y, p);
        project<MU, SF>(p, h);
        store6(to_lower, nface, f, h);
    }
    {
        const int y = face_site<MU>(g, f, g.L[MU] - 1, c);
        cx<float> p[12], h[6], u[6], r2[3], w[6];
        P32::load_spinor(in, nullptr, g.V, y, p);
        project<MU, SB>(p, h);
        P32::load_link(U, g.V, MU, y, u, r2);
        su3_adj_mul(u, r2, h, 1.0f, w);
        store6(to_upper, nface, f, w);
    }
}

__device__ __forceinline__ bool on_cut_face(const Geom &g, const HaloGeom &hg, const int c[4])
{
    bool s = false;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if ((hg.split_mask >> m) & 1) s |= c[m] == 0 || c[m] == g.L[m] - 1;
    return s;
}

// in: the sites with no hop across a cut face
template <int KIND>
__global__ void __launch_bounds__(kHaloThreads) k_apply_interior(Geom g, HaloGeom hg, GaugeStore U, CloverStore C,
                                                                 const void *in, void *out, double kappa)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    int c[4];
    site_coords(g, x, c);
    if (on_cut_face(g, hg, c)) return;
    apply_site_at<P32, KIND>(g, x, U, C, in, nullptr, out, nullptr, kappa);
}

// the hops of direction MU of a surface site: from the local field, or from
// the received buffers across a cut face (the same arithmetic as hop_dir)
template <int MU, int SF, int SB>
__device__ __forceinline__ void hop_dir_halo(const Geom &g, const HaloGeom &hg, const HaloBufs &hb,
                                             const GaugeStore &U, const void *in, int x, const int c[4], float k,
                                             cx<float> acc[12])
{
    if (!((hg.split_mask >> MU) & 1)) {
        hop_dir<P32, MU, SF, SB>(g, U, in, nullptr, x, c, k, acc);
        return;
    }
    const int L = g.L[MU], st = g.stride[MU];
    {
        cx<float> h[6], u[6], r2[3], w[6];
        float coef = k;
        if (c[MU] == L - 1) {
            load6(hb.from_upper[MU], hg.nface[MU], face_index<MU>(g, c), h);
            if (MU == 3 && hg.fwd_cross_t) coef = k * (float)g.tbc;
        } else {
            cx<float> p[12];
            P32::load_spinor(in, nullptr, g.V, x + st, p);
            project<MU, SF>(p, h);
        }
        P32::load_link(U, g.V, MU, x, u, r2);
        su3_mul(u, r2, h, coef, w);
        reconstruct_add<MU, SF>(acc, w);
    }
    {
        cx<float> w[6];
        if (c[MU] == 0) {
            cx<float> y[6];
            load6(hb.from_lower[MU], hg.nface[MU], face_index<MU>(g, c), y);
            const float coef = (MU == 3 && hg.bwd_cross_t) ? k * (float)g.tbc : k;
#pragma unroll
            for (int j = 0; j < 6; ++j) w[j] = coef * y[j];
        } else {
            const int xb = x - st;
            cx<float> p[12], h[6], u[6], r2[3];
            P32::load_spinor(in, nullptr, g.V, xb, p);
            project<MU, SB>(p, h);
            P32::load_link(U, g.V, MU, xb, u, r2);
            su3_adj_mul(u, r2, h, k, w);
        }
        reconstruct_add<MU, SB>(acc, w);
    }
}

// post: the sites on cut faces.  Thread i walks the faces of the cut
// directions in order (direction mu: nface lower-face sites, then nface
// upper-face sites); a site on the faces of several cut directions is
// computed by the thread of the first of them.
template <int KIND>
__global__ void __launch_bounds__(kHaloThreads) k_apply_surface(Geom g, HaloGeom hg, HaloBufs hb, GaugeStore U,
                                                                CloverStore C, const void *in, void *out,
                                                                double kappa, int nthreads)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nthreads) return;
    int mu = 0;
    for (; mu < 4; ++mu) {
        if (!((hg.split_mask >> mu) & 1)) continue;
        if (i < 2 * hg.nface[mu]) break;
        i -= 2 * hg.nface[mu];
    }
    if (mu == 4) return;
    const int f = i % hg.nface[mu], upper = i / hg.nface[mu];
    int c[4], x;
    switch (mu) {
    case 0: x = face_site<0>(g, f, upper ? g.L[0] - 1 : 0, c); break;
    case 1: x = face_site<1>(g, f, upper ? g.L[1] - 1 : 0, c); break;
    case 2: x = face_site<2>(g, f, upper ? g.L[2] - 1 : 0, c); break;
    default: x = face_site<3>(g, f, upper ? g.L[3] - 1 : 0, c); break;
    }
    for (int m = 0; m < mu; ++m)
        if (((hg.split_mask >> m) & 1) && (c[m] == 0 || c[m] == g.L[m] - 1)) return;
    // the rest as apply_site_at: clover on the centre spinor, then the hops
    cx<float> acc[12];
    {
        cx<float> p[12];
        P32::load_spinor(in, nullptr, g.V, x, p);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            float r[36];
            P32::load_clover(C, g.V, x, b, r);
            clover_block_mul(r, p + 6 * b, acc + 6 * b);
        }
    }
    const float k = (float)(-kappa);
    constexpr int SF = KIND == 1 ? +1 : -1;
    constexpr int SB = -SF;
    hop_dir_halo<0, SF, SB>(g, hg, hb, U, in, x, c, k, acc);
    hop_dir_halo<1, SF, SB>(g, hg, hb, U, in, x, c, k, acc);
    hop_dir_halo<2, SF, SB>(g, hg, hb, U, in, x, c, k, acc);
    hop_dir_halo<3, SF, SB>(g, hg, hb, U, in, x, c, k, acc);
    P32::store_spinor(out, nullptr, g.V, x, acc);
}

// extended-lattice site of local site x (one halo site across every cut face)
__device__ __forceinline__ int ext_site(const Geom &gl, const Geom &ge, int split_mask, int x)
{
    int c[4];
    site_coords(gl, x, c);
    int e = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) e += (c[m] + ((split_mask >> m) & 1)) * ge.stride[m];
    return e;
}

template <class T>
__global__ void k_extract(Geom gl, Geom ge, int split_mask, const T *src, T *dst, int nplanes)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nplanes * gl.V) return;
    const int x = (int)(i % gl.V), p = (int)(i / gl.V);
    dst[(size_t)p * gl.V + x] = src[(size_t)p * ge.V + ext_site(gl, ge, split_mask, x)];
}

template <class T>
cudaError_t extract(const wc_lattice_s *sub, const T *src, T *dst, int nplanes, cudaStream_t stream)
{
    const long long n = (long long)nplanes * sub->g.V;
    k_extract<T><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(sub->g, sub->ext->g, sub->split_mask, src, dst,
                                                                   nplanes);
    return cudaGetLastError();
}

HaloGeom halo_geom(const wc_lattice_s *lat)
{
    HaloGeom h;
    h.split_mask = lat->split_mask;
    for (int m = 0; m < 4; ++m) h.nface[m] = lat->g.V / lat->g.L[m];
    h.fwd_cross_t = lat->offset[3] + lat->g.L[3] == lat->global_L[3];
    h.bwd_cross_t = lat->offset[3] == 0;
    return h;
}

wc_status check_subdomain_fields(wc_lattice lat, wc_field out, wc_field in)
{
    if (!lat) return set_error(nullptr, WC_ERR_ARG, "lattice is NULL");
    if (!lat->split_mask) return set_error(lat, WC_ERR_ARG, "not a sub-domain lattice (wc_create_subdomain)");
    if (!in || in->lat != lat || (out && out->lat != lat))
        return set_error(lat, WC_ERR_ARG, "fields must belong to the sub-domain");
    if (in->prec != WC_F32 || (out && out->prec != WC_F32))
        return set_error(lat, WC_ERR_ARG, "the decomposed operator works on FP32 fields");
    if (out && (out == in || out->data == in->data)) return set_error(lat, WC_ERR_ARG, "out and in must be distinct");
    if (!lat->gauge_loaded || !lat->clover_loaded) return set_error(lat, WC_ERR_STATE, "gauge/clover not loaded");
    return WC_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

cudaError_t extract_gauge(wc_lattice sub, cudaStream_t stream)
{
    const GaugeStore &s = sub->ext->gauge;
    GaugeStore &d = sub->gauge;
    cudaError_t e = extract(sub, s.u64, d.u64, 36, stream);
    if (e == cudaSuccess) e = extract(sub, s.udf, d.udf, 36, stream);
    if (e == cudaSuccess) e = extract(sub, s.u32, d.u32, 12, stream);
    if (e == cudaSuccess) e = extract(sub, s.u16a, d.u16a, 4, stream);
    if (e == cudaSuccess) e = extract(sub, s.u16b, d.u16b, 4, stream);
    return e;
}

cudaError_t extract_clover(wc_lattice sub, cudaStream_t stream)
{
    const CloverStore &s = sub->ext->clover;
    CloverStore &d = sub->clover;
    cudaError_t e = extract(sub, s.c64, d.c64, 36, stream);
    if (e == cudaSuccess) e = extract(sub, s.cdf, d.cdf, 36, stream);
    if (e == cudaSuccess) e = extract(sub, s.c32, d.c32, 18, stream);
    if (e == cudaSuccess) e = extract(sub, s.c16, d.c16, 9, stream);
    return e;
}

}  // namespace wc

using namespace wc;

extern "C" {

wc_status wc_create_subdomain(const int local_dims[4], const int global_dims[4], const int offset[4], int t_bc,
                              void *cuda_stream, wc_lattice *out)
{
    if (!local_dims || !global_dims || !offset || !out)
        return set_error(nullptr, WC_ERR_ARG, "local_dims, global_dims, offset and out must not be NULL");
    *out = nullptr;
    int mask = 0, ext_dims[4];
    for (int m = 0; m < 4; ++m) {
        if (local_dims[m] < 2 || global_dims[m] < local_dims[m])
            return set_error(nullptr, WC_ERR_ARG, "need 2 <= local extent <= global extent in every direction");
        if (offset[m] < 0 || offset[m] + local_dims[m] > global_dims[m])
            return set_error(nullptr, WC_ERR_ARG, "the sub-domain must lie inside the global lattice");
        if (local_dims[m] < global_dims[m]) mask |= 1 << m;
        ext_dims[m] = local_dims[m] + (((mask >> m) & 1) ? 2 : 0);
    }
    if (!mask) return set_error(nullptr, WC_ERR_ARG, "no direction is cut: use wc_create_lattice");
    wc_lattice lat = nullptr;
    wc_status st = wc_create_lattice(local_dims, t_bc, cuda_stream, &lat);
    if (st != WC_OK) return st;
    wc_lattice ext = nullptr;
    st = wc_create_lattice(ext_dims, t_bc, cuda_stream, &ext);
    if (st != WC_OK) {
        wc_destroy_lattice(lat);
        return st;
    }
    for (int m = 0; m < 4; ++m) {
        lat->global_L[m] = global_dims[m];
        lat->offset[m] = offset[m];
    }
    lat->split_mask = mask;
    lat->ext = ext;
    *out = lat;
    return WC_OK;
}

wc_status wc_halo_bytes(wc_lattice lat, int mu, long long *bytes)
{
    if (!lat || !bytes || mu < 0 || mu > 3) return set_error(lat, WC_ERR_ARG, "lattice, bytes and 0 <= mu < 4 needed");
    *bytes = ((lat->split_mask >> mu) & 1) ? (long long)(lat->g.V / lat->g.L[mu]) * 3 * sizeof(float4) : 0;
    return WC_OK;
}

wc_status wc_halo_pack(wc_lattice lat, wc_field in, int dagger, void *const send[8])
{
    wc_status st = check_subdomain_fields(lat, nullptr, in);
    if (st != WC_OK) return st;
    if (!send) return set_error(lat, WC_ERR_ARG, "send is NULL");
    for (int m = 0; m < 4; ++m)
        if ((lat->split_mask >> m) & 1)
            for (int d = 0; d < 2; ++d)
                if (!send[2 * m + d] || !aligned16(send[2 * m + d]))
                    return set_error(lat, WC_ERR_ARG, "send buffers of cut directions must be 16-byte aligned device memory");
    const Geom &g = lat->g;
    for (int m = 0; m < 4; ++m) {
        if (!((lat->split_mask >> m) & 1)) continue;
        const int nface = g.V / g.L[m];
        const unsigned grid = (nface + kHaloThreads - 1) / kHaloThreads;
        float4 *lo = static_cast<float4 *>(send[2 * m]), *up = static_cast<float4 *>(send[2 * m + 1]);
        const int sf = dagger ? 1 : -1;
#define WC_PACK(MU)                                                                                            \
    if (sf < 0)                                                                                                \
        k_halo_pack<MU, -1><<<grid, kHaloThreads, 0, lat->stream>>>(g, nface, lat->gauge, in->data, lo, up); \
    else                                                                                                       \
        k_halo_pack<MU, +1><<<grid, kHaloThreads, 0, lat->stream>>>(g, nface, lat->gauge, in->data, lo, up);
        switch (m) {
        case 0: WC_PACK(0) break;
        case 1: WC_PACK(1) break;
        case 2: WC_PACK(2) break;
        default: WC_PACK(3) break;
        }
#undef WC_PACK
        st = check_launch(lat, "halo_pack");
        if (st != WC_OK) return st;
    }
    return WC_OK;
}

wc_status wc_apply_interior(wc_lattice lat, wc_field out, wc_field in, int dagger)
{
    if (!out) return set_error(lat, WC_ERR_ARG, "out is NULL");
    wc_status st = check_subdomain_fields(lat, out, in);
    if (st != WC_OK) return st;
    const HaloGeom hg = halo_geom(lat);
    const unsigned grid = (lat->g.V + kHaloThreads - 1) / kHaloThreads;
    if (dagger)
        k_apply_interior<1><<<grid, kHaloThreads, 0, lat->stream>>>(lat->g, hg, lat->gauge, lat->clover, in->data,
                                                                    out->data, lat->kappa);
    else
        k_apply_interior<0><<<grid, kHaloThreads, 0, lat->stream>>>(lat->g, hg, lat->gauge, lat->clover, in->data,
                                                                    out->data, lat->kappa);
    return check_launch(lat, "apply_interior");
}

wc_status wc_apply_surface(wc_lattice lat, wc_field out, wc_field in, int dagger, const void *const recv[8])
{
    if (!out) return set_error(lat, WC_ERR_ARG, "out is NULL");
    wc_status st = check_subdomain_fields(lat, out, in);
    if (st != WC_OK) return st;
    if (!recv) return set_error(lat, WC_ERR_ARG, "recv is NULL");
    HaloBufs hb{};
    int n = 0;
    const HaloGeom hg = halo_geom(lat);
    for (int m = 0; m < 4; ++m) {
        if (!((lat->split_mask >> m) & 1)) continue;
        for (int d = 0; d < 2; ++d)
            if (!recv[2 * m + d] || !aligned16(recv[2 * m + d]))
                return set_error(lat, WC_ERR_ARG, "receive buffers of cut directions must be 16-byte aligned device memory");
        hb.from_lower[m] = static_cast<const float4 *>(recv[2 * m]);
        hb.from_upper[m] = static_cast<const float4 *>(recv[2 * m + 1]);
        n += 2 * hg.nface[m];
    }
    const unsigned grid = (n + kHaloThreads - 1) / kHaloThreads;
    if (dagger)
        k_apply_surface<1><<<grid, kHaloThreads, 0, lat->stream>>>(lat->g, hg, hb, lat->gauge, lat->clover, in->data,
                                                                   out->data, lat->kappa, n);
    else
        k_apply_surface<0><<<grid, kHaloThreads, 0, lat->stream>>>(lat->g, hg, hb, lat->gauge, lat->clover, in->data,
                                                                   out->data, lat->kappa, n);
    return check_launch(lat, "apply_surface");
}

}  // extern "C"
