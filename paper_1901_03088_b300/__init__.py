"""B300-native (sm_103a) improved structure-preserving colour normalisation
(SPCN) for H&E pathology images, after Ramakrishnan, Anand & Sethi,
arXiv 1901.03088.

    from paper_1901_03088_b300 import spcn     # loads libspcn.so (CUDA)
    ctx = spcn.Context(0)
    st_src = ctx.estimate_basis(src)            # basis, i0, sampled P99
    st_tgt = ctx.estimate_basis(tgt)
    st_tgt.p99[:] = ctx.stain_percentile(tgt, st_tgt)   # exact target P99
    out = ctx.normalize(src, st_src, st_tgt)

``synth`` holds the seeded synthetic-slide generators used by the tests and
the benchmark.  Importing the package itself loads nothing.
"""
