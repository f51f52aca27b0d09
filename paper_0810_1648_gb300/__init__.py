"""GaBP SVM solver (Bickson, Yom-Tov, Dolev) on one GB300: CUDA hot path behind a C ABI."""
