// Mixed form, 3D: the node kernels of the mesh step that march along i3 (2.5D blocking).
// A block owns a 32 x 8 column of the (i1, i2) plane and a chunk of zc planes of it.  The
// planes it reads (its nodes plus a one-node halo in i1 and i2) sit in a ring of shared-memory
// planes: the ghost maps of the boundary conditions are applied once, when a plane is staged,
// and every node value is loaded once per pass plus the halo, so the stencil arithmetic runs
// without boundary branches.  A sweep's arithmetic per node is that of jacobi_y_kernel, term
// for term; the filter sums filter_kernel's weights one direction at a time.
#include "es_mesh.cuh"

namespace es {

// Theta at node (g0, g1, g2), which lies at most one node outside the grid in one direction:
// the map of s_map at a ghost node.  Other positions (outside in two directions, or further
// out) are no face neighbour of any node of the grid and read as zero.
__device__ __forceinline__ float m3_theta(const Inst& I, const float* __restrict__ th, int g0, int g1, int g2)
{
    const int n0 = I.n[0], n1 = I.n[1], n2 = I.n[2];
    const bool o0 = g0 < 0 || g0 >= n0, o1 = g1 < 0 || g1 >= n1, o2 = g2 < 0 || g2 >= n2;
    if (g0 < -1 || g0 > n0 || g1 < -1 || g1 > n1 || g2 < -1 || g2 > n2 || (int)o0 + (int)o1 + (int)o2 > 1) return 0.0f;
    if (!(o0 || o1 || o2)) return th[((long long)g2 * n1 + g1) * n0 + g0];
    return th[s_map(I, g0, g1, g2)];
}

// Mesh spacings of the mixed Jacobi sweeps, stored once per edge: E_k[j] at node i is
// x^n_j(i + e_k) - x^n_j(i) formed in FP64 and rounded to binary32, on the grid extended by
// one node below in every direction (entry i_k = -1 is the edge from the ghost node to the
// first node).  The sweep reads dl_{k+}(i) = E_k(i) and dl_{k-}(i) = -E_k(i - e_k): rounding
// to nearest is symmetric, so the negated entry is the rounded difference taken the other way.
// Rows have the pitch e3_pitch and node i1 = 0 sits at column 4 (es_mesh.cuh).
struct Edges3 {
    long long ne;                 // entries per component: pitch (n1 + 1)(n2 + 1)
    int x0, x1;                   // row pitch, rows per plane (n1 + 1)
    __device__ explicit Edges3(const Inst& I) : x0(e3_pitch(I.n[0])), x1(I.n[1] + 1)
    {
        ne = (long long)x0 * x1 * (I.n[2] + 1);
    }
    __device__ long long at(int g0, int g1, int g2) const
    {
        return ((long long)(g2 + 1) * x1 + (g1 + 1)) * x0 + (g0 + 4);
    }
};

// the three components of E_k at node g from the 9-layer ghost-extended positions XE
__device__ __forceinline__ void m3_edge_xe(const Inst& I, const double* __restrict__ XE, int k, int g0, int g1,
                                           int g2, float e[3])
{
    const long long X0 = I.n[0] + 18, X1 = I.n[1] + 18, nx = X0 * X1 * (I.n[2] + 18);
    const long long c = ((long long)(g2 + 9) * X1 + (g1 + 9)) * X0 + (g0 + 9);
    const long long s = k == 0 ? 1 : (k == 1 ? X0 : X0 * X1);
#pragma unroll
    for (int j = 0; j < 3; ++j) e[j] = f64_to_f32(XE[j * nx + c + s] - XE[j * nx + c]);
}

// E_k of plane q at this thread's node (k = 0, 1, 2), E_0 left of its row (lane 0) and E_1
// below its column's first row (warp 0), formed from XE; zero where no node is, and all zero
// unless act.  Each entry is stored once: a node's own edges, and the edges from the ghost
// nodes below the grid where the column touches the low boundary.
__device__ __forceinline__ void m3_edges(const Inst& I, const Scratch& Sc, const Edges3& EG, const Col3& C, int g0,
                                         int g1, int q, bool act, float ep[3][3], float e0h[3], float e1h[3])
{
    float* E = Sc.dl;
    const bool valid = act && g0 < I.n[0] && g1 < I.n[1];
    const bool left = act && g0 == C.b0 && g1 < I.n[1], below = act && g1 == C.b1 && g0 < I.n[0];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        e0h[j] = 0.0f;
        e1h[j] = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) ep[k][j] = 0.0f;
    }
    if (valid) {
        const long long e = EG.at(g0, g1, q);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            m3_edge_xe(I, Sc.XE, k, g0, g1, q, ep[k]);
#pragma unroll
            for (int j = 0; j < 3; ++j) E[(k * 3 + j) * EG.ne + e] = ep[k][j];
        }
    }
    if (left) {
        m3_edge_xe(I, Sc.XE, 0, C.b0 - 1, g1, q, e0h);
        if (C.b0 == 0) {
#pragma unroll
            for (int j = 0; j < 3; ++j) E[j * EG.ne + EG.at(-1, g1, q)] = e0h[j];
        }
    }
    if (below) {
        m3_edge_xe(I, Sc.XE, 1, g0, C.b1 - 1, q, e1h);
        if (C.b1 == 0) {
#pragma unroll
            for (int j = 0; j < 3; ++j) E[(3 + j) * EG.ne + EG.at(g0, -1, q)] = e1h[j];
        }
    }
}

// E_2 of the plane below the chunk (the minus-i3 spacing of the chunk's first plane), formed
// from XE and stored where it is the edge from the ghost plane below the grid
__device__ __forceinline__ void m3_edge_below(const Inst& I, const Scratch& Sc, const Edges3& EG, int g0, int g1,
                                              int z0, float e[3])
{
    e[0] = e[1] = e[2] = 0.0f;
    if (g0 >= I.n[0] || g1 >= I.n[1]) return;
    m3_edge_xe(I, Sc.XE, 2, g0, g1, z0 - 1, e);
    if (z0 == 0) {
        const long long a = EG.at(g0, g1, -1);
#pragma unroll
        for (int j = 0; j < 3; ++j) Sc.dl[(6 + j) * EG.ne + a] = e[j];
    }
}

// The first mixed Jacobi sweep of a 3D instance, with the arithmetic of jacobi_y_kernel:
// y_i <- sum_{k,s} w_{k,s} (dl_{k,s} + y_{i+-e_k}) / sum_{k,s} w_{k,s}, w_{k,s} = (Theta_i +
// Theta_{i+-e_k}) / 2 / dxi_k^2, in the order k = 1, 2, 3 with the minus side first, from
// y = 0.  It forms the spacings from XE (x^n with its ghost maps, staged by the metrics pass
// that opens the mesh step) and stores them for the later sweeps.  Theta sits in a ring of
// four staged planes, loaded one plane ahead.  LAST (a single sweep): the limiter bounds of
// Sec. 4, dl_{k,s}[k] / (2 y_k) with s the sign of y_k, reduced to the instance minimum.
template <bool LAST>
__global__ void __launch_bounds__(NODE_TPB, 3) jacobi3d_first_kernel(const Inst* __restrict__ insts,
                                                                      const int2* __restrict__ work, int nwork,
                                                                      const Scratch* __restrict__ scr, int theta_sel)
{
    pdl_entry();
    __shared__ float sth[4][M3_PY][M3_PX];
    __shared__ float se1[2][3][M3_TY][M3_TX];
    __shared__ double sh[32];
    const int lx = (int)threadIdx.x % M3_TX, ly = (int)threadIdx.x / M3_TX;
    int ha = -1, hb = -1;
    if ((int)threadIdx.x < M3_NH) m3_halo_slot((int)threadIdx.x, ha, hb);
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        const Scratch& Sc = scr[it.x];
        const Col3 C = col3(I, it.y);
        const Edges3 EG(I);
        const long long n = I.ncell;
        const float* th = reinterpret_cast<const float*>(theta_sel ? Sc.th1 : Sc.th0);
        float* yd = reinterpret_cast<float*>(Sc.xa);     // the sweep count starts at 0
        const int g0 = C.b0 + lx, g1 = C.b1 + ly, h0 = C.b0 - 1 + ha, h1 = C.b1 - 1 + hb;
        const bool valid = g0 < I.n[0] && g1 < I.n[1];
        __syncthreads();    // the previous item's readers of the ring are done
        // planes z0 - 1, z0 and z0 + 1 into the ring (z0 + 1 <= z1: the plane above the chunk
        // is a grid plane or the ghost plane i3 = n3)
        for (int q = C.z0 - 1; q <= C.z0 + 1; ++q) {
            const int s = q & 3;
            sth[s][ly + 1][lx + 1] = m3_theta(I, th, g0, g1, q);
            if (ha >= 0) sth[s][hb][ha] = m3_theta(I, th, h0, h1, q);
        }
        float ep[3][3], e0h[3], e1h[3], em2[3];
        m3_edges(I, Sc, EG, C, g0, g1, C.z0, true, ep, e0h, e1h);
        m3_edge_below(I, Sc, EG, g0, g1, C.z0, em2);
        float bnd = 1.0f;
        for (int z = C.z0; z < C.z1; ++z) {
#pragma unroll
            for (int j = 0; j < 3; ++j) se1[z & 1][j][ly][lx] = ep[1][j];
            __syncthreads();
            // loads of the next planes: Theta of plane z + 2, the edges of plane z + 1
            const bool more = z + 2 <= C.z1;
            float to = 0.0f, tv = 0.0f;
            if (more) {
                to = m3_theta(I, th, g0, g1, z + 2);
                if (ha >= 0) tv = m3_theta(I, th, h0, h1, z + 2);
            }
            float epn[3][3], e0n[3], e1n[3];
            m3_edges(I, Sc, EG, C, g0, g1, z + 1, z + 1 < C.z1, epn, e0n, e1n);
            // the minus-side spacings of this node: E_0 of the left neighbour (the lane
            // before), E_1 of the node below (the row before), E_2 of the plane below
            float em[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const float l = __shfl_up_sync(0xffffffffu, ep[0][j], 1);
                em[0][j] = lx == 0 ? e0h[j] : l;
                em[1][j] = ly == 0 ? e1h[j] : se1[z & 1][j][ly - 1][lx];
                em[2][j] = em2[j];
            }
            if (valid) {
                const int c = z & 3, m = (z - 1) & 3, pp = (z + 1) & 3;
                const float tc = sth[c][ly + 1][lx + 1];
                const float tn[3][2] = { { sth[c][ly + 1][lx], sth[c][ly + 1][lx + 2] },
                                         { sth[c][ly][lx + 1], sth[c][ly + 2][lx + 1] },
                                         { sth[m][ly + 1][lx + 1], sth[pp][ly + 1][lx + 1] } };
                float num[3] = { 0.0f, 0.0f, 0.0f }, den = 0.0f, dk[3][2];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const float w = 0.5f * (tc + tn[k][s]) * I.f_h2[k];
                        float dv[3], yv[3];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            dv[j] = s ? ep[k][j] : -em[k][j];
                            yv[j] = 0.0f;
                        }
                        dk[k][s] = dv[k];
#pragma unroll
                        for (int j = 0; j < 3; ++j) num[j] = fmaf(w, dv[j] + yv[j], num[j]);
                        den += w;
                    }
                float ynew[3];
                const long long p = ((long long)z * I.n[1] + g1) * I.n[0] + g0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    ynew[j] = num[j] / den;
                    yd[j * n + p] = ynew[j];
                }
                if (LAST) {
                    float b = 1.0f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float dx = ynew[k];
                        if (dx < 0.0f) b = fminf(b, dk[k][0] / (2.0f * dx));
                        else if (dx > 0.0f) b = fminf(b, dk[k][1] / (2.0f * dx));
                    }
                    if (!(b >= 0.0f)) b = 0.0f;
                    bnd = fminf(bnd, b);
                }
            }
            // plane z + 2 into the ring: its slot last held plane z - 2, read at plane z - 1
            if (more) {
                const int s = (z + 2) & 3;
                sth[s][ly + 1][lx + 1] = to;
                if (ha >= 0) sth[s][hb][ha] = tv;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                em2[j] = ep[2][j];
                e0h[j] = e0n[j];
                e1h[j] = e1n[j];
#pragma unroll
                for (int k = 0; k < 3; ++k) ep[k][j] = epn[k][j];
            }
        }
        if (LAST) {
            const double mb = block_min_pos(f32_to_f64(bnd), sh);
            if (threadIdx.x == 0) atomic_min_pos(&Sc.red[5], mb);
        }
    }
}

// asynchronous 4-byte global -> shared copies (cp.async) and their groups
__device__ __forceinline__ void m3_cp4(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void m3_cp16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void m3_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void m3_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// the grid node whose Theta and y a staged position g stands for (g at most one node outside
// the grid, in one direction) and the component of y that a wall mirror negates there (-1:
// none).  At one node outside, the mirror of y_at and the copy of s_map pick the same node
// (the boundary node), and a periodic side wraps for both.  False: g is no face neighbour
// of a grid node.
__device__ __forceinline__ bool m3_source(const Inst& I, int g0, int g1, int g2, long long& src, int& flip)
{
    int i[3] = { g0, g1, g2 }, out = 0;
    flip = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int n = I.n[k];
        if (i[k] < -1 || i[k] > n) return false;
        if (i[k] >= 0 && i[k] < n) continue;
        ++out;
        const int side = i[k] < 0 ? 0 : 1;
        if (I.bc[k][side] == BC_PERIODIC) {
            i[k] = side == 0 ? n - 1 : 0;
        } else {
            i[k] = side == 0 ? 0 : n - 1;
            flip = k;
        }
    }
    if (out > 1) return false;
    src = ((long long)i[2] * I.n[1] + i[1]) * I.n[0] + i[0];
    return true;
}

// shared memory of the later sweeps: Theta and y planes in a ring of six (three read by a
// plane's update, two in flight, one spare), the spacings E_k of a plane (this column's nodes,
// the E_0 left of each row, the E_1 below the first row) in a ring of four
constexpr int J3_YR = 6, J3_ER = 4;
struct J3Smem {
    float y[J3_YR][3][M3_PY][M3_PX];
    float th[J3_YR][M3_PY][M3_PX];
    alignas(16) float e[J3_ER][9][M3_TY][M3_TX];
    float e0h[J3_ER][3][M3_TY];
    alignas(16) float e1h[J3_ER][3][M3_TX];
};

// A later Jacobi sweep of a 3D instance (the arithmetic of jacobi3d_first_kernel with y read
// from the previous sweep, bit for bit that of jacobi_y_kernel).  The planes are staged with
// cp.async two planes ahead of the update: at plane i3 each thread waits for the copies it
// issued two planes before (Theta and y up to plane i3 + 1, the spacings of plane i3), and
// after the block barrier the block issues Theta and y of plane i3 + 3 and the spacings of
// plane i3 + 2.  A thread that copied a ghost position across a wall negates the mirrored
// component of y after its copy lands, before the barrier.
template <bool LAST>
__global__ void __launch_bounds__(NODE_TPB, 3) jacobi3d_async_kernel(const Inst* __restrict__ insts,
                                                                      const int2* __restrict__ work, int nwork,
                                                                      const Scratch* __restrict__ scr, int sweep,
                                                                      int theta_sel)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char m3_dyn[];
    J3Smem& S = *reinterpret_cast<J3Smem*>(m3_dyn);
    __shared__ double sh[32];
    const int lx = (int)threadIdx.x % M3_TX, ly = (int)threadIdx.x / M3_TX;
    int ha = -1, hb = -1;
    if ((int)threadIdx.x < M3_NH) m3_halo_slot((int)threadIdx.x, ha, hb);
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        const Scratch& Sc = scr[it.x];
        const Col3 C = col3(I, it.y);
        const Edges3 EG(I);
        const long long n = I.ncell;
        const float* th = reinterpret_cast<const float*>(theta_sel ? Sc.th1 : Sc.th0);
        const float* ys = reinterpret_cast<const float*>(sweep % 2 == 1 ? Sc.xa : Sc.xb);
        float* yd = reinterpret_cast<float*>(sweep % 2 == 0 ? Sc.xa : Sc.xb);
        const float* E = Sc.dl;
        const int g0 = C.b0 + lx, g1 = C.b1 + ly;
        const bool valid = g0 < I.n[0] && g1 < I.n[1];
        // a staged position inside the grid reads its own node; only ghost positions need the
        // boundary maps
        auto inside = [&](int s0, int s1, int q) {
            return (unsigned)s0 < (unsigned)I.n[0] && (unsigned)s1 < (unsigned)I.n[1] && (unsigned)q < (unsigned)I.n[2];
        };
        // Theta and y of plane q at this thread's position and halo position
        auto stage_y = [&](int q) {
            const int r = (q + J3_YR) % J3_YR;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && ha < 0) break;
                const int a = h ? ha : lx + 1, b = h ? hb : ly + 1;
                const int s0 = C.b0 - 1 + a, s1 = C.b1 - 1 + b;
                long long src;
                int fl;
                if (inside(s0, s1, q)) src = ((long long)q * I.n[1] + s1) * I.n[0] + s0;
                else if (!m3_source(I, s0, s1, q, src, fl)) continue;
                m3_cp4(&S.th[r][b][a], th + src);
#pragma unroll
                for (int j = 0; j < 3; ++j) m3_cp4(&S.y[r][j][b][a], ys + j * n + src);
            }
        };
        // after the copies of plane q landed: the wall mirror's sign
        auto fix_y = [&](int q) {
            const int r = (q + J3_YR) % J3_YR;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && ha < 0) break;
                const int a = h ? ha : lx + 1, b = h ? hb : ly + 1;
                const int s0 = C.b0 - 1 + a, s1 = C.b1 - 1 + b;
                long long src;
                int fl;
                if (inside(s0, s1, q) || !m3_source(I, s0, s1, q, src, fl) || fl < 0) continue;
                S.y[r][fl][b][a] = -S.y[r][fl][b][a];
            }
        };
        // the spacings of plane q (k0 = 2: only E_2, for the plane below the chunk): each row of
        // the column in 16-byte copies, the E_0 left of each row in 4-byte copies
        auto stage_e = [&](int q, int k0) {
            const int r = q & (J3_ER - 1);
            const int t = (int)threadIdx.x;
            const long long e0 = EG.at(C.b0, C.b1, q);
            for (int c = t; c < (9 - 3 * k0) * M3_TY * 8; c += NODE_TPB) {
                const int kj = 3 * k0 + c / (M3_TY * 8), row = (c / 8) % M3_TY, seg = c % 8;
                if (C.b1 + row >= I.n[1]) continue;
                m3_cp16(&S.e[r][kj][row][4 * seg], E + kj * EG.ne + e0 + (long long)row * EG.x0 + 4 * seg);
            }
            if (k0 > 0) return;
            if (t < M3_TY && C.b1 + t < I.n[1]) {
                const long long e = EG.at(C.b0 - 1, C.b1 + t, q);
#pragma unroll
                for (int j = 0; j < 3; ++j) m3_cp4(&S.e0h[r][j][t], E + j * EG.ne + e);
            } else if (t >= 32 && t < 32 + 3 * 8) {
                const int j = (t - 32) / 8, seg = (t - 32) % 8;
                m3_cp16(&S.e1h[r][j][4 * seg], E + (3 + j) * EG.ne + EG.at(C.b0, C.b1 - 1, q) + 4 * seg);
            }
        };
        __syncthreads();    // the previous item's readers of the rings are done
        for (int q = C.z0 - 1; q <= C.z0 + 1; ++q) stage_y(q);
        stage_e(C.z0 - 1, 2);
        stage_e(C.z0, 0);
        m3_commit();
        if (C.z0 + 2 <= C.z1) stage_y(C.z0 + 2);
        if (C.z0 + 1 < C.z1) stage_e(C.z0 + 1, 0);
        m3_commit();
        float bnd = 1.0f;
        for (int z = C.z0; z < C.z1; ++z) {
            m3_wait<1>();    // this thread's copies for plane z (y: up to z + 1) have landed
            if (z == C.z0) {
                fix_y(z - 1);
                fix_y(z);
            }
            fix_y(z + 1);
            __syncthreads();
            if (z + 3 <= C.z1) stage_y(z + 3);
            if (z + 2 < C.z1) stage_e(z + 2, 0);
            m3_commit();
            if (valid) {
                const int c = (z + J3_YR) % J3_YR, m = (z - 1 + J3_YR) % J3_YR, pp = (z + 1) % J3_YR;
                const int ec = z & (J3_ER - 1), em_ = (z - 1) & (J3_ER - 1);
                float ep[3][3], em[3][3];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) ep[k][j] = S.e[ec][k * 3 + j][ly][lx];
                    em[0][j] = lx == 0 ? S.e0h[ec][j][ly] : S.e[ec][j][ly][lx - 1];
                    em[1][j] = ly == 0 ? S.e1h[ec][j][lx] : S.e[ec][3 + j][ly - 1][lx];
                    em[2][j] = S.e[em_][6 + j][ly][lx];
                }
                const float tc = S.th[c][ly + 1][lx + 1];
                const float tn[3][2] = { { S.th[c][ly + 1][lx], S.th[c][ly + 1][lx + 2] },
                                         { S.th[c][ly][lx + 1], S.th[c][ly + 2][lx + 1] },
                                         { S.th[m][ly + 1][lx + 1], S.th[pp][ly + 1][lx + 1] } };
                float num[3] = { 0.0f, 0.0f, 0.0f }, den = 0.0f, dk[3][2];
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const float w = 0.5f * (tc + tn[k][s2]) * I.f_h2[k];
                        float dv[3], yv[3];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            dv[j] = s2 ? ep[k][j] : -em[k][j];
                            yv[j] = k == 0 ? S.y[c][j][ly + 1][lx + 2 * s2]
                                  : (k == 1 ? S.y[c][j][ly + 2 * s2][lx + 1] : S.y[s2 ? pp : m][j][ly + 1][lx + 1]);
                        }
                        dk[k][s2] = dv[k];
#pragma unroll
                        for (int j = 0; j < 3; ++j) num[j] = fmaf(w, dv[j] + yv[j], num[j]);
                        den += w;
                    }
                float ynew[3];
                const long long p = ((long long)z * I.n[1] + g1) * I.n[0] + g0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    ynew[j] = num[j] / den;
                    yd[j * n + p] = ynew[j];
                }
                if (LAST) {
                    float b = 1.0f;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float dx = ynew[k];
                        if (dx < 0.0f) b = fminf(b, dk[k][0] / (2.0f * dx));
                        else if (dx > 0.0f) b = fminf(b, dk[k][1] / (2.0f * dx));
                    }
                    if (!(b >= 0.0f)) b = 0.0f;
                    bnd = fminf(bnd, b);
                }
            }
        }
        m3_wait<0>();
        if (LAST) {
            const double mb = block_min_pos(f32_to_f64(bnd), sh);
            if (threadIdx.x == 0) atomic_min_pos(&Sc.red[5], mb);
        }
    }
}

void prepare_mesh3d()
{
    cudaFuncSetAttribute(jacobi3d_async_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(J3Smem));
    cudaFuncSetAttribute(jacobi3d_async_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(J3Smem));
}

void launch_jacobi3d(bool first, bool last, int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork,
                     const Scratch* scr, int sweep, int theta_sel)
{
    const size_t sm = sizeof(J3Smem);
    if (first) {
        if (last) pdl_launch(jacobi3d_first_kernel<true>, grid, NODE_TPB, 0, st, insts, work, nwork, scr, theta_sel);
        else pdl_launch(jacobi3d_first_kernel<false>, grid, NODE_TPB, 0, st, insts, work, nwork, scr, theta_sel);
    } else {
        if (last) pdl_launch(jacobi3d_async_kernel<true>, grid, NODE_TPB, sm, st, insts, work, nwork, scr, sweep, theta_sel);
        else pdl_launch(jacobi3d_async_kernel<false>, grid, NODE_TPB, sm, st, insts, work, nwork, scr, sweep, theta_sel);
    }
}

// the halo slots with the four corners (h in [0, M3_NH + 4)): the 3 x 3 stencils need them
__device__ __forceinline__ void m3_halo_slot_c(int h, int& a, int& b)
{
    if (h < M3_NH) { m3_halo_slot(h, a, b); return; }
    a = (h - M3_NH) % 2 == 0 ? 0 : M3_PX - 1;
    b = h - M3_NH < 2 ? 0 : M3_PY - 1;
}

// a scalar node field at (g0, g1, g2) within one node of the grid in every direction, through
// the map of s_map (periodic wrap, else the boundary node); zero further out
__device__ __forceinline__ float m3_scalar(const Inst& I, const float* __restrict__ f, int g0, int g1, int g2)
{
    const int n0 = I.n[0], n1 = I.n[1], n2 = I.n[2];
    if (g0 < -1 || g0 > n0 || g1 < -1 || g1 > n1 || g2 < -1 || g2 > n2) return 0.0f;
    if (g0 >= 0 && g0 < n0 && g1 >= 0 && g1 < n1 && g2 >= 0 && g2 < n2) return f[((long long)g2 * n1 + g1) * n0 + g0];
    return f[s_map(I, g0, g1, g2)];
}

// One pass of the low-pass filter on a 3D instance (mixed form): the 3^3 stencil with weights
// (1/2)^(|j|_1 + 3), the tensor product of (1/4, 1/2, 1/4) in each direction, taken one
// direction at a time: rows r(j2) = (a(i1-1) + a(i1+1)) / 4 + a(i1) / 2 of a staged plane,
// the plane sums P = (r(-1) + r(1)) / 4 + r(0) / 2, then (P(i3-1) + P(i3+1)) / 4 + P(i3) / 2.
// Each plane sum serves three output planes.  Ghost nodes of the stencil: the maps of s_map.
__global__ void __launch_bounds__(NODE_TPB) filter3d_kernel(const Inst* __restrict__ insts,
                                                             const int2* __restrict__ work, int nwork,
                                                             const Scratch* __restrict__ scr, int parity)
{
    pdl_entry();
    __shared__ float sa[2][M3_PY][M3_PX];
    const int lx = (int)threadIdx.x % M3_TX, ly = (int)threadIdx.x / M3_TX;
    int ha = -1, hb = -1;
    if ((int)threadIdx.x < M3_NH + 4) m3_halo_slot_c((int)threadIdx.x, ha, hb);
    for (int wi = blockIdx.x; wi < nwork; wi += gridDim.x) {
        const int2 it = work[wi];
        const Inst& I = insts[it.x];
        const Scratch& Sc = scr[it.x];
        const Col3 C = col3(I, it.y);
        const float* a = reinterpret_cast<const float*>(parity ? Sc.th1 : Sc.th0);
        float* dst = reinterpret_cast<float*>(parity ? Sc.th0 : Sc.th1);
        const int g0 = C.b0 + lx, g1 = C.b1 + ly, h0 = C.b0 - 1 + ha, h1 = C.b1 - 1 + hb;
        const bool valid = g0 < I.n[0] && g1 < I.n[1];
        __syncthreads();    // the previous item's readers are done
        float vo = m3_scalar(I, a, g0, g1, C.z0 - 1), vh = ha >= 0 ? m3_scalar(I, a, h0, h1, C.z0 - 1) : 0.0f;
        float pm2 = 0.0f, pm1 = 0.0f;
        for (int q = C.z0 - 1; q <= C.z1; ++q) {
            const int b = q & 1;
            sa[b][ly + 1][lx + 1] = vo;
            if (ha >= 0) sa[b][hb][ha] = vh;
            __syncthreads();
            if (q < C.z1) {
                vo = m3_scalar(I, a, g0, g1, q + 1);
                if (ha >= 0) vh = m3_scalar(I, a, h0, h1, q + 1);
            }
            float r[3];
#pragma unroll
            for (int j = 0; j < 3; ++j)
                r[j] = 0.25f * (sa[b][ly + j][lx] + sa[b][ly + j][lx + 2]) + 0.5f * sa[b][ly + j][lx + 1];
            const float pq = 0.25f * (r[0] + r[2]) + 0.5f * r[1];
            if (valid && q >= C.z0 + 1)
                dst[((long long)(q - 1) * I.n[1] + g1) * I.n[0] + g0] = 0.25f * (pm2 + pq) + 0.5f * pm1;
            pm2 = pm1;
            pm1 = pq;
        }
    }
}

void launch_filter3d(int grid, cudaStream_t st, const Inst* insts, const int2* work, int nwork, const Scratch* scr,
                     int parity)
{
    pdl_launch(filter3d_kernel, grid, NODE_TPB, 0, st, insts, work, nwork, scr, parity);
}

}  // namespace es
