"""Edge clustering of dynamic graphs via the weighted line-graph skeleton
(arXiv 2311.10337) on one GB300 (sm_103a): hand-written CUDA kernels behind
the C ABI of include/dgec.h, driven through the ctypes binding `dgec`.

    import numpy as np, torch
    from paper_2311_10337_gb300 import dgec

    ctx = dgec.Context(0)
    # temporal edges (i, j, t): int32 src/dst, int64 t, on the GPU
    out = ctx.run(src, dst, t, n_vertices, k=8, min_cluster_size=5)
    labels = out.numpy("labels")            # edge clusters, -1 = noise
    forest = out.numpy("mst_w")             # also sk_*, knn_id, core, link_*, cl_*
    # from host arrays, copies included
    labels, n_clusters = ctx.run_host(src_np, dst_np, t_np, n_vertices, 8, 5)
    # Alg. 5 at thresholds omega; time cutoff / nearly-causal variants of Sec. 4.3
    lv = ctx.run_levels(src, dst, t, n_vertices, [2 ** i for i in range(29)], 5)
    out = ctx.run(src, dst, t, n_vertices, 8, 5, delta_max=3600)
    out = ctx.run(src, dst, t, n_vertices, 8, 5, delta_nc=60)
    # many graphs in one pass, hypergraphs (Sec. 4.4), a serving loop
    ctx.run_batch(...); ctx.run_hyper(...); dgec.Server(...)

Every call runs on the GPU; there is no CPU path. `synth` holds the seeded
workload generators.
"""
