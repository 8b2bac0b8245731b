"""FP64 brute-force CPU oracle of the radar scan and CPU references of the
LBVH build steps.  Test infrastructure only: never imported by the product
package."""
