// extern "C" entry points of libmeshrast (declared in include/meshrast.h):
// argument checks, workspace layout and the launch sequence of each call.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "meshrast.h"
#include "rast_common.cuh"
#include "rast_internal.h"

namespace mr_host {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool ws_layout(const rast_params *p, int64_t V, int64_t F, mr::WsLayout *L) {
    (void)V;
    std::memset(L, 0, sizeof(*L));
    size_t off = 0;
    L->status = 0;
    L->queue = 4;
    L->total = 8;
    L->maxcount = 16;
    L->redo = 20;
    L->redo_q = 24;
    L->redo_head = 28;
    off = 256;
    L->records = off;
    off = align256(off + (size_t)F * sizeof(mr::FaceRec));
    L->face_mesh = off;
    off = align256(off + (size_t)F * sizeof(int));
    if (p->bin_size > 0) {
        const int64_t nb = (p->image_size + p->bin_size - 1) / p->bin_size;
        const int64_t NB = (int64_t)p->N * nb * nb;
        const int64_t cap = p->max_bin_entries > 0 ? p->max_bin_entries : NB * (int64_t)p->max_faces_per_bin;
        L->nb = nb;
        L->NB = NB;
        L->capacity = cap;
        L->counts = off;
        off = align256(off + (size_t)NB * 4);
        L->eff = off;
        off = align256(off + (size_t)NB * 4);
        L->offsets = off;
        off = align256(off + (size_t)(NB + 1) * 4);
        L->cursor = off;
        off = align256(off + (size_t)NB * 4);
        L->order = off;
        off = align256(off + (size_t)NB * 4);
        if (p->faces_per_pixel > 16) {
            // the streaming pass's queue: one entry per 8 x 4 block at most
            L->redo_items = off;
            off = align256(off + (size_t)NB * (size_t)(p->bin_size * p->bin_size / 32) * 8);
        }
        L->lists = off;
        off = align256(off + (size_t)cap * 8);
    }
    L->bytes = off;
    return true;
}

int num_sms() {
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    std::call_once(once[dev], [dev]() {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    });
    return cached[dev];
}

static bool check_params(const rast_params *p, int64_t V, int64_t F) {
    if (!p) return false;
    if (p->N < 0 || p->N > 65535 || p->image_size < 1 || p->image_size > 8192) return false;
    if (p->faces_per_pixel < 1) return false;
    if (!(p->blur_radius >= 0.f) || !(p->blur_radius < 4.f)) return false;
    if (p->perspective_correct != 0 && p->perspective_correct != 1) return false;
    if (p->clip_barycentric_coords != 0 && p->clip_barycentric_coords != 1) return false;
    if (p->reserved != 0 || p->reserved_f != 0.f) return false;
    if (V < 0 || F < 0 || F >= 0x7fffffffLL || V >= 0x7fffffffLL) return false;
    if (p->bin_size > 0 && p->max_faces_per_bin <= 0) return false;
    if (p->max_bin_entries < 0) return false;
    return true;
}

static int unsupported(const rast_params *p) {
    if (p->faces_per_pixel > mr::kMaxK) return 1;
    if (p->bin_size != 0 && p->bin_size != 8 && p->bin_size != 16) return 1;
    if (p->bin_size > 0) {
        // bin keys, counts, offsets and list positions are 32-bit on the device:
        // refuse layouts that would not fit instead of clamping them
        const int64_t nb = (p->image_size + p->bin_size - 1) / p->bin_size;
        const int64_t NB = (int64_t)p->N * nb * nb;
        if (NB >= 0x7fffffffLL) return 1;
        const int64_t cap = p->max_bin_entries > 0 ? p->max_bin_entries : NB * (int64_t)p->max_faces_per_bin;
        if (cap > 0x7fffffffLL) return 1;
    }
    return 0;
}

}  // namespace mr_host

using mr::WsLayout;

extern "C" {

size_t rast_workspace_bytes(const rast_params *p, int64_t V, int64_t F) {
    if (!mr_host::check_params(p, V, F) || mr_host::unsupported(p)) return 0;
    WsLayout L;
    mr_host::ws_layout(p, V, F, &L);
    return L.bytes;
}

static int stage(const rast_params *p, const float *verts, int64_t V, const int64_t *faces, int64_t F,
                 const int64_t *first_face, const int64_t *num_faces, const float *cams, char *ws,
                 const WsLayout &L, int do_count, cudaStream_t st) {
    mr::StageArgs a;
    a.verts = verts;
    a.V = V;
    a.faces = faces;
    a.F = F;
    a.first_face = first_face;
    a.num_faces = num_faces;
    a.N = p->N;
    a.cams = cams;
    a.blur = p->blur_radius;
    a.S = p->image_size;
    a.bin = p->bin_size > 0 ? p->bin_size : 1;
    a.nb = (int)L.nb;
    a.do_count = do_count;
    a.rec = reinterpret_cast<mr::FaceRec *>(ws + L.records);
    a.face_mesh = reinterpret_cast<int *>(ws + L.face_mesh);
    a.counts = do_count ? reinterpret_cast<int *>(ws + L.counts) : nullptr;
    a.status = reinterpret_cast<unsigned *>(ws + L.status);
    return mr::launch_stage(a, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

static int check_ws(const rast_params *p, int64_t V, int64_t F, void *ws, size_t ws_bytes, WsLayout *L) {
    mr_host::ws_layout(p, V, F, L);
    if (!ws || ((uintptr_t)ws & 255u) != 0 || ws_bytes < L->bytes) return MESHRAST_ERR_WORKSPACE;
    return MESHRAST_OK;
}

// Forward rasterization; with `blend` set, the fine pass also applies the blend
// (register path, K <= 16) and *blended tells whether it did.
static int forward(const rast_params *p, const float *verts, int64_t V, const int64_t *faces, int64_t F,
                   const int64_t *first_face, const int64_t *num_faces, const float *cams, int64_t *pix_to_face,
                   float *zbuf, float *bary, float *dists, void *workspace, size_t workspace_bytes, void *stream,
                   const mr::FineBlend *blend, bool *blended) {
    if (blended) *blended = false;
    if (!mr_host::check_params(p, V, F)) return MESHRAST_ERR_INVALID_ARG;
    if (mr_host::unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    if (p->N > 0 && (!first_face || !num_faces || !cams)) return MESHRAST_ERR_INVALID_ARG;
    if (F > 0 && (!faces || (V > 0 && !verts))) return MESHRAST_ERR_INVALID_ARG;
    const int64_t S = p->image_size, K = p->faces_per_pixel;
    const int64_t slots = (int64_t)p->N * S * S * K;
    const bool binned = p->bin_size > 0;
    // no Fragment data at all: only when the fine pass itself blends the silhouette
    const bool no_frag = !pix_to_face && !zbuf && !bary && !dists;
    const bool fine_blend = blend && binned && mr::fine_blends((int)K, blend->rgb != 0);
    if (slots > 0 && (!pix_to_face || !zbuf || !bary || !dists) && !(no_frag && fine_blend))
        return MESHRAST_ERR_INVALID_ARG;
    WsLayout L;
    int rc = check_ws(p, V, F, workspace, workspace_bytes, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    if (cudaMemsetAsync(ws, 0, 256, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    if (p->N == 0) return MESHRAST_OK;
    if (binned && L.NB > 0) {
        if (cudaMemsetAsync(ws + L.counts, 0, (size_t)L.NB * 4, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    }
    rc = stage(p, verts, V, faces, F, first_face, num_faces, cams, ws, L, binned ? 1 : 0, st);
    if (rc) return rc;
    mr::EvalFlags fl;
    fl.persp = p->perspective_correct;
    fl.clip = p->clip_barycentric_coords;
    fl.blur = p->blur_radius;
    fl.znear = 0.f;  // set per image below for the plain form; binned: per-face check at staging
    mr::FineOut out{pix_to_face, zbuf, bary, dists};
    if (!binned) {
        mr::NaiveArgs a;
        a.rec = reinterpret_cast<const mr::FaceRec *>(ws + L.records);
        a.cams = cams;
        a.first_face = first_face;
        a.num_faces = num_faces;
        a.F = F;
        a.S = (int)S;
        a.K = (int)K;
        a.fl = fl;
        a.out = out;
        return mr::launch_naive(a, p->N, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
    }
    // Large K: the front-to-back streaming fine pass, when every bin's list is
    // sorted as one piece (capacity <= 8192) and a candidate's depth is never
    // below its face's nearest corner (clipped barycentrics, or no blur);
    // Fragment attributes (and the silhouette blend) in a pass of their own.
    const bool zcull = p->clip_barycentric_coords || !(p->blur_radius > 0.f);
    // (work items: 32-pixel blocks of every bin, counted by a 32-bit queue)
    const bool items_fit = L.NB * (int64_t)(p->bin_size * p->bin_size / 32) < 0x7fffffffLL;
    const bool streaming =
        K > 16 && zcull && p->max_faces_per_bin <= 8192 && items_fit && pix_to_face && zbuf && bary && dists;
    // The block fine pass takes bins longest first.  The streaming pass keeps
    // the natural (image, bin) order: its items are small, and consecutive
    // items of one image keep that image's face records and lists in L2.
    int *const order = streaming ? nullptr : reinterpret_cast<int *>(ws + L.order);
    mr::ScanArgs sa;
    sa.counts = reinterpret_cast<const int *>(ws + L.counts);
    sa.eff = reinterpret_cast<int *>(ws + L.eff);
    sa.offsets = reinterpret_cast<int *>(ws + L.offsets);
    sa.cursor = reinterpret_cast<int *>(ws + L.cursor);
    sa.order = order;
    sa.NB = L.NB;
    sa.capacity = L.capacity;
    sa.max_per_bin = p->max_faces_per_bin;
    sa.queue = reinterpret_cast<unsigned *>(ws + L.queue);
    sa.status = reinterpret_cast<unsigned *>(ws + L.status);
    sa.total = reinterpret_cast<long long *>(ws + L.total);
    sa.maxcount = reinterpret_cast<int *>(ws + L.maxcount);
    sa.first_face = first_face;
    sa.num_faces = num_faces;
    sa.N = p->N;
    sa.F = F;
    if (mr::launch_scan(sa, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    mr::FillArgs fa;
    fa.rec = reinterpret_cast<const mr::FaceRec *>(ws + L.records);
    fa.face_mesh = reinterpret_cast<const int *>(ws + L.face_mesh);
    fa.F = F;
    fa.S = (int)S;
    fa.bin = p->bin_size;
    fa.nb = (int)L.nb;
    fa.cursor = reinterpret_cast<int *>(ws + L.cursor);
    fa.eff = reinterpret_cast<const int *>(ws + L.eff);
    fa.offsets = reinterpret_cast<const int *>(ws + L.offsets);
    fa.lists = reinterpret_cast<unsigned long long *>(ws + L.lists);
    if (mr::launch_fill(fa, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    mr::FineArgs ka;
    ka.rec = reinterpret_cast<const mr::FaceRec *>(ws + L.records);
    ka.cams = cams;
    ka.lists = reinterpret_cast<unsigned long long *>(ws + L.lists);
    ka.eff = reinterpret_cast<const int *>(ws + L.eff);
    ka.offsets = reinterpret_cast<const int *>(ws + L.offsets);
    ka.order = order;
    ka.queue = reinterpret_cast<unsigned *>(ws + L.queue);
    ka.redo_count = reinterpret_cast<unsigned *>(ws + L.redo);
    ka.redo_q = reinterpret_cast<unsigned *>(ws + L.redo_q);
    ka.redo_head = reinterpret_cast<unsigned *>(ws + L.redo_head);
    ka.redo_items = L.redo_items ? reinterpret_cast<unsigned long long *>(ws + L.redo_items) : nullptr;
    ka.items = (int)L.NB;
    ka.nb = (int)L.nb;
    ka.S = (int)S;
    ka.K = (int)K;
    ka.fl = fl;
    ka.out = out;
    std::memset(&ka.blend, 0, sizeof(ka.blend));
    if (streaming) {
        int cap = 256;
        while (cap < p->max_faces_per_bin) cap <<= 1;
        ka.sort_cap = cap;
        if (mr::launch_fine_stream(ka, p->bin_size, st) != cudaSuccess) return MESHRAST_ERR_CUDA;
        mr::FragAttrArgs fa2;
        fa2.rec = ka.rec;
        fa2.out = out;
        fa2.F = F;
        fa2.status = reinterpret_cast<unsigned *>(ws + L.status);
        fa2.P = (int64_t)p->N * S * S;
        fa2.S = (int)S;
        fa2.K = (int)K;
        fa2.fl = fl;
        fa2.sigma = blend ? blend->sigma : 1.f;
        fa2.image = (blend && !blend->rgb) ? blend->image : nullptr;
        if (fa2.image && blended) *blended = true;
        return mr::launch_frag_attr(fa2, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
    }
    ka.sort_cap = mr::fine_sort_cap(p->max_faces_per_bin, (int)K, p->bin_size * p->bin_size);
    if (fine_blend) {
        ka.blend = *blend;
        ka.blend.frag = no_frag ? 0 : 1;
        if (blended) *blended = true;
    }
    return mr::launch_fine(ka, p->bin_size, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int rast_mesh_fwd(const rast_params *p, const float *verts, int64_t V, const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces, const float *cams, int64_t *pix_to_face,
                  float *zbuf, float *bary, float *dists, void *workspace, size_t workspace_bytes, void *stream) {
    return forward(p, verts, V, faces, F, first_face, num_faces, cams, pix_to_face, zbuf, bary, dists, workspace,
                   workspace_bytes, stream, nullptr, nullptr);
}

int rast_mesh_bwd(const rast_params *p, const float *verts, int64_t V, const int64_t *faces, int64_t F,
                  const int64_t *first_face, const int64_t *num_faces, const float *cams,
                  const int64_t *pix_to_face, const float *grad_zbuf, const float *grad_bary,
                  const float *grad_dists, float *grad_verts, void *workspace, size_t workspace_bytes,
                  void *stream) {
    if (!mr_host::check_params(p, V, F)) return MESHRAST_ERR_INVALID_ARG;
    if (mr_host::unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    if (p->N > 0 && (!first_face || !num_faces || !cams)) return MESHRAST_ERR_INVALID_ARG;
    if (F > 0 && (!faces || (V > 0 && !verts))) return MESHRAST_ERR_INVALID_ARG;
    if (V > 0 && !grad_verts) return MESHRAST_ERR_INVALID_ARG;
    const int64_t S = p->image_size, K = p->faces_per_pixel;
    const int64_t slots = (int64_t)p->N * S * S * K;
    if (slots > 0 && !pix_to_face) return MESHRAST_ERR_INVALID_ARG;
    WsLayout L;
    int rc = check_ws(p, V, F, workspace, workspace_bytes, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    if (V > 0 && cudaMemsetAsync(grad_verts, 0, (size_t)V * 3 * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (slots == 0 || (!grad_zbuf && !grad_bary && !grad_dists)) return MESHRAST_OK;
    rc = stage(p, verts, V, faces, F, first_face, num_faces, cams, ws, L, 0, st);
    if (rc) return rc;
    mr::RastBwdArgs a;
    a.rec = reinterpret_cast<const mr::FaceRec *>(ws + L.records);
    a.face_mesh = reinterpret_cast<const int *>(ws + L.face_mesh);
    a.faces = faces;
    a.verts = verts;
    a.cams = cams;
    a.pix_to_face = pix_to_face;
    a.grad_zbuf = grad_zbuf;
    a.grad_bary = grad_bary;
    a.grad_dists = grad_dists;
    a.grad_verts = grad_verts;
    a.F = F;
    a.V = V;
    a.slots = slots;
    a.S = (int)S;
    a.K = (int)K;
    a.fl.persp = p->perspective_correct;
    a.fl.clip = p->clip_barycentric_coords;
    a.fl.blur = p->blur_radius;
    a.fl.znear = 0.f;
    return mr::launch_rast_bwd(a, p->N, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

static int check_blend(const blend_params *bp, int64_t N, int64_t S, int64_t K) {
    if (!bp) return MESHRAST_ERR_INVALID_ARG;
    if (N < 0 || N > 65535 || S < 0 || S > 8192 || K < 1 || K > mr::kMaxK)
        return K > mr::kMaxK ? MESHRAST_ERR_UNSUPPORTED : MESHRAST_ERR_INVALID_ARG;
    if (!(bp->sigma > 0.f) || !(bp->gamma > 0.f) || !(bp->zfar > bp->znear)) return MESHRAST_ERR_INVALID_ARG;
    if (bp->mode != MESHRAST_BLEND_SIL && bp->mode != MESHRAST_BLEND_RGB) return MESHRAST_ERR_INVALID_ARG;
    if (bp->reserved != 0) return MESHRAST_ERR_INVALID_ARG;
    return MESHRAST_OK;
}

static void fill_blend(mr::BlendArgs &a, const blend_params *bp, int64_t N, int64_t S, int64_t K,
                       const int64_t *pix_to_face, const float *zbuf, const float *bary, const float *dists,
                       const int64_t *faces, int64_t F, const float *colors, int64_t V) {
    std::memset(&a, 0, sizeof(a));
    a.P = N * S * S;
    a.N = (int)N;
    a.S = (int)S;
    a.F = F;
    a.V = V;
    a.K = (int)K;
    a.pix_to_face = pix_to_face;
    a.zbuf = zbuf;
    a.bary = bary;
    a.dists = dists;
    a.faces = faces;
    a.colors = colors;
    a.sigma = bp->sigma;
    a.gamma = bp->gamma;
    a.znear = bp->znear;
    a.zfar = bp->zfar;
    a.eps = bp->eps;
    a.bg0 = bp->bg[0];
    a.bg1 = bp->bg[1];
    a.bg2 = bp->bg[2];
    a.mode = bp->mode;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

int blend_fwd(const blend_params *bp, int64_t N, int64_t S, int64_t K, const int64_t *pix_to_face,
              const float *zbuf, const float *bary, const float *dists, const int64_t *faces, int64_t F,
              const float *vert_colors, int64_t V, float *image, void *stream) {
    int rc = check_blend(bp, N, S, K);
    if (rc) return rc;
    const int64_t P = N * S * S;
    if (P == 0) return MESHRAST_OK;
    if (!pix_to_face || !dists || !image) return MESHRAST_ERR_INVALID_ARG;
    if (bp->mode == MESHRAST_BLEND_RGB && (!zbuf || !bary || !faces || !vert_colors || F < 0 || V < 0))
        return MESHRAST_ERR_INVALID_ARG;
    if (!aligned16(image) || !aligned16(pix_to_face) || !aligned16(dists) || (zbuf && !aligned16(zbuf)))
        return MESHRAST_ERR_INVALID_ARG;
    mr::BlendArgs a;
    fill_blend(a, bp, N, S, K, pix_to_face, zbuf, bary, dists, faces, F, vert_colors, V);
    a.image = image;
    return mr::launch_blend_fwd(a, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? MESHRAST_OK
                                                                                          : MESHRAST_ERR_CUDA;
}

int rast_blend_fwd(const rast_params *p, const blend_params *bp, const float *verts, int64_t V,
                   const int64_t *faces, int64_t F, const int64_t *first_face, const int64_t *num_faces,
                   const float *cams, const float *vert_colors, int64_t *pix_to_face, float *zbuf, float *bary,
                   float *dists, float *image, void *workspace, size_t workspace_bytes, void *stream) {
    if (!mr_host::check_params(p, V, F)) return MESHRAST_ERR_INVALID_ARG;
    if (mr_host::unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    const int64_t N = p->N, S = p->image_size, K = p->faces_per_pixel;
    int rc = check_blend(bp, N, S, K);
    if (rc) return rc;
    const bool rgb = bp->mode == MESHRAST_BLEND_RGB;
    const int64_t P = N * S * S;
    const bool no_frag = !pix_to_face && !zbuf && !bary && !dists;
    if (P > 0) {
        if (!image || !aligned16(image)) return MESHRAST_ERR_INVALID_ARG;
        if (no_frag) {
            // silhouette without Fragment data: only where the fine pass blends
            if (rgb || p->bin_size == 0 || !mr::fine_blends((int)K, false)) return MESHRAST_ERR_INVALID_ARG;
        } else if (!pix_to_face || !dists || !aligned16(pix_to_face) || !aligned16(dists) ||
                   (zbuf && !aligned16(zbuf))) {
            return MESHRAST_ERR_INVALID_ARG;
        }
        if (rgb && (!faces || !vert_colors)) return MESHRAST_ERR_INVALID_ARG;
    }
    mr::FineBlend fbl;
    std::memset(&fbl, 0, sizeof(fbl));
    fbl.on = 1;
    fbl.rgb = rgb ? 1 : 0;
    fbl.sigma = bp->sigma;
    fbl.gamma = bp->gamma;
    fbl.znear = bp->znear;
    fbl.zfar = bp->zfar;
    fbl.eps = bp->eps;
    fbl.bg0 = bp->bg[0];
    fbl.bg1 = bp->bg[1];
    fbl.bg2 = bp->bg[2];
    fbl.faces = faces;
    fbl.colors = vert_colors;
    fbl.F = F;
    fbl.V = V;
    fbl.image = image;
    bool blended = false;
    rc = forward(p, verts, V, faces, F, first_face, num_faces, cams, pix_to_face, zbuf, bary, dists, workspace,
                 workspace_bytes, stream, &fbl, &blended);
    if (rc || blended || P == 0) return rc;
    // the plain form and K > 16: the blend kernel on the written fragments
    mr::BlendArgs a;
    fill_blend(a, bp, N, S, K, pix_to_face, zbuf, bary, dists, faces, F, vert_colors, V);
    a.image = image;
    return mr::launch_blend_fwd(a, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess ? MESHRAST_OK
                                                                                          : MESHRAST_ERR_CUDA;
}

int blend_bwd(const blend_params *bp, int64_t N, int64_t S, int64_t K, const int64_t *pix_to_face,
              const float *zbuf, const float *bary, const float *dists, const int64_t *faces, int64_t F,
              const float *vert_colors, int64_t V, const float *grad_image, float *grad_zbuf, float *grad_bary,
              float *grad_dists, float *grad_vert_colors, void *stream) {
    int rc = check_blend(bp, N, S, K);
    if (rc) return rc;
    const int64_t P = N * S * S;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const bool rgb = bp->mode == MESHRAST_BLEND_RGB;
    if (rgb) {
        if (!faces || !vert_colors || !grad_vert_colors || F < 0 || V < 0) return MESHRAST_ERR_INVALID_ARG;
        if (V > 0 && cudaMemsetAsync(grad_vert_colors, 0, (size_t)V * 3 * sizeof(float), st) != cudaSuccess)
            return MESHRAST_ERR_CUDA;
    }
    if (P == 0) return MESHRAST_OK;
    if (!pix_to_face || !dists || !grad_image || !grad_dists) return MESHRAST_ERR_INVALID_ARG;
    if (rgb && (!zbuf || !bary || !grad_zbuf || !grad_bary)) return MESHRAST_ERR_INVALID_ARG;
    if (!aligned16(grad_image) || !aligned16(pix_to_face) || !aligned16(dists) || !aligned16(grad_dists) ||
        (zbuf && !aligned16(zbuf)))
        return MESHRAST_ERR_INVALID_ARG;
    mr::BlendArgs a;
    fill_blend(a, bp, N, S, K, pix_to_face, zbuf, bary, dists, faces, F, vert_colors, V);
    a.grad_image = grad_image;
    a.grad_zbuf = grad_zbuf;
    a.grad_bary = grad_bary;
    a.grad_dists = grad_dists;
    a.grad_colors = grad_vert_colors;
    return mr::launch_blend_bwd(a, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int blend_rast_bwd(const rast_params *p, const blend_params *bp, const float *verts, int64_t V,
                   const int64_t *faces, int64_t F, const int64_t *first_face, const int64_t *num_faces,
                   const float *cams, const int64_t *pix_to_face, const float *zbuf, const float *bary,
                   const float *dists, const float *vert_colors, const float *grad_image, float *grad_verts,
                   float *grad_vert_colors, void *workspace, size_t workspace_bytes, void *stream) {
    if (!mr_host::check_params(p, V, F)) return MESHRAST_ERR_INVALID_ARG;
    if (mr_host::unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    const int64_t N = p->N, S = p->image_size, K = p->faces_per_pixel;
    int rc = check_blend(bp, N, S, K);
    if (rc) return rc;
    const bool rgb = bp->mode == MESHRAST_BLEND_RGB;
    if (N > 0 && (!first_face || !num_faces || !cams)) return MESHRAST_ERR_INVALID_ARG;
    if (F > 0 && (!faces || (V > 0 && !verts))) return MESHRAST_ERR_INVALID_ARG;
    if (V > 0 && !grad_verts) return MESHRAST_ERR_INVALID_ARG;
    if (rgb && (!faces || !vert_colors || (V > 0 && !grad_vert_colors))) return MESHRAST_ERR_INVALID_ARG;
    const int64_t slots = N * S * S * K;
    if (slots > 0) {
        if (!pix_to_face || !dists || !grad_image) return MESHRAST_ERR_INVALID_ARG;
        if (rgb && (!zbuf || !bary)) return MESHRAST_ERR_INVALID_ARG;
        if (!aligned16(grad_image) || !aligned16(pix_to_face) || !aligned16(dists) || (zbuf && !aligned16(zbuf)))
            return MESHRAST_ERR_INVALID_ARG;
    }
    WsLayout L;
    rc = check_ws(p, V, F, workspace, workspace_bytes, &L);
    if (rc) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char *ws = reinterpret_cast<char *>(workspace);
    if (V > 0 && cudaMemsetAsync(grad_verts, 0, (size_t)V * 3 * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (rgb && V > 0 && cudaMemsetAsync(grad_vert_colors, 0, (size_t)V * 3 * sizeof(float), st) != cudaSuccess)
        return MESHRAST_ERR_CUDA;
    if (slots == 0) return MESHRAST_OK;
    rc = stage(p, verts, V, faces, F, first_face, num_faces, cams, ws, L, 0, st);
    if (rc) return rc;
    mr::BlendArgs a;
    fill_blend(a, bp, N, S, K, pix_to_face, zbuf, bary, dists, faces, F, vert_colors, V);
    a.grad_image = grad_image;
    a.grad_colors = grad_vert_colors;
    mr::RastBwdArgs r;
    std::memset(&r, 0, sizeof(r));
    r.rec = reinterpret_cast<const mr::FaceRec *>(ws + L.records);
    r.face_mesh = reinterpret_cast<const int *>(ws + L.face_mesh);
    r.faces = faces;
    r.verts = verts;
    r.cams = cams;
    r.pix_to_face = pix_to_face;
    r.grad_verts = grad_verts;
    r.F = F;
    r.V = V;
    r.slots = slots;
    r.S = (int)S;
    r.K = (int)K;
    r.fl.persp = p->perspective_correct;
    r.fl.clip = p->clip_barycentric_coords;
    r.fl.blur = p->blur_radius;
    r.fl.znear = 0.f;
    return mr::launch_blend_rast_bwd(a, r, st) == cudaSuccess ? MESHRAST_OK : MESHRAST_ERR_CUDA;
}

int rast_query_status(const void *workspace, uint32_t *status, void *stream) {
    if (!workspace || !status) return MESHRAST_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    uint32_t v = 0;
    if (cudaMemcpy(&v, workspace, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return MESHRAST_ERR_CUDA;
    *status = v;
    return MESHRAST_OK;
}

int rast_bin_occupancy(const rast_params *p, int64_t V, int64_t F, const void *workspace, int32_t *max_count,
                       int64_t *total_entries, void *stream) {
    if (!mr_host::check_params(p, V, F) || !workspace || !max_count || !total_entries)
        return MESHRAST_ERR_INVALID_ARG;
    if (p->bin_size <= 0) return MESHRAST_ERR_INVALID_ARG;
    WsLayout L;
    mr_host::ws_layout(p, V, F, &L);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return MESHRAST_ERR_CUDA;
    const char *ws = reinterpret_cast<const char *>(workspace);
    int32_t mc = 0;
    long long tot = 0;
    if (cudaMemcpy(&mc, ws + L.maxcount, 4, cudaMemcpyDeviceToHost) != cudaSuccess) return MESHRAST_ERR_CUDA;
    if (cudaMemcpy(&tot, ws + L.total, 8, cudaMemcpyDeviceToHost) != cudaSuccess) return MESHRAST_ERR_CUDA;
    *max_count = mc;
    *total_entries = tot;
    return MESHRAST_OK;
}

int rast_workspace_bin_layout(const rast_params *p, int64_t V, int64_t F, rast_bin_layout *out) {
    if (!out || !mr_host::check_params(p, V, F)) return MESHRAST_ERR_INVALID_ARG;
    if (mr_host::unsupported(p)) return MESHRAST_ERR_UNSUPPORTED;
    if (p->bin_size <= 0) return MESHRAST_ERR_INVALID_ARG;
    WsLayout L;
    mr_host::ws_layout(p, V, F, &L);
    out->counts = (int64_t)L.counts;
    out->eff = (int64_t)L.eff;
    out->offsets = (int64_t)L.offsets;
    out->lists = (int64_t)L.lists;
    out->nb = L.nb;
    out->NB = L.NB;
    out->capacity = L.capacity;
    out->bytes = (int64_t)L.bytes;
    out->redo = (int64_t)L.redo;
    out->order = (int64_t)L.order;
    return MESHRAST_OK;
}

const char *rast_strerror(int code) {
    switch (code) {
        case MESHRAST_OK: return "ok";
        case MESHRAST_ERR_INVALID_ARG: return "invalid argument";
        case MESHRAST_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
        case MESHRAST_ERR_UNSUPPORTED:
            return "unsupported parameters (K > 64, bin_size not in {0, 8, 16}, or 2^31 - 1 or more bins or bin-list "
                   "entries)";
        case MESHRAST_ERR_CUDA: return "CUDA launch failed";
        case MESHRAST_ERR_STATIC_TOO_LARGE:
            return "the call needs more workspace than the library's built-in 16 MiB array (use rast_mesh_fwd)";
        default: return "unknown error";
    }
}

}  // extern "C"
